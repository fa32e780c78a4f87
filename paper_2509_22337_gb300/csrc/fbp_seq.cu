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
//   A. every new a->v message of the level from the messages as they stand
//      (all reads before any write, as the level's sequential order allows),
//      one warp per edge, staged in shared memory;
//   B. after one block barrier, together: the writes (factor-major messages
//      and the variable-major copy), and the beliefs of the touched rows.  A
//      row of degree <= 8 (one thread) and each touched 32-entry sub-chunk of
//      a longer row (one warp) read their entries and replace those written
//      in this level by the staged values (the host lists them), so they
//      need not wait for the writes; their loads are issued before step A,
//      whose work hides them.  The warp that recomputes a row's only
//      touched sub-chunk also finishes the row: a row of 2..8 sub-chunks
//      from its products, a longer (hub) row by updating one slot chain and
//      the eight butterfly nodes above it, kept per hub row;
//   C. only where a row had several touched sub-chunks: after a barrier, the
//      row recombined whole.
// A message read in step A thus includes every update of the earlier levels,
// as in the in-place sequential execution of a schedule's levels (Sec. 4.3).  Levels are short (about ten edges on BINGO-1M SEQFIX), so the
// whole run is one block of kFloodSlots threads.  Every product is grouped as
// in the flooding kernels (sub-chunks multiplied in order, 256 slots, the xor
// butterfly), so a belief kept current here has the bits a flooding phase 1
// would compute from the same messages.
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

constexpr int kTreeNodes = 2 * kFloodSlots;  // per hub row: node (k, j) of butterfly level k at k + j; leaves at 256..511

struct SeqHalfDev {
    int32_t n_levels;
    const int32_t *lp, *le;  // level starts; level edges
    const int4 *dp;          // [n_levels + 1] starts of {short items, sub-chunk items, whole medium rows, whole hub rows}
    const int4 *ds;          // short-row items {variable, patch begin, patch end, 0}
    const int4 *dk;          // sub-chunk items {sub-chunk, patch begin, patch end, finish}
    const int32_t *dm, *dh;  // rows with several touched sub-chunks, recombined whole
    const int2 *pt;          // patches {position in the row or sub-chunk, index in the level}
};

struct SeqArgs {
    DevGraph g;
    FloodPlanDev F;
    float *a2v;                        // factor-major messages, updated in place
    float *a2v_vm;                     // variable-major copy
    float *tmp;                        // new messages of a level wider than the shared stage
    XP *tree;                          // [n_hub_rows * kTreeNodes] butterfly nodes of every hub row
    SeqHalfDev half[2];
    int32_t n_halves;
    int32_t max_iters;
    float tol;
    unsigned *res;                     // [max_iters] residual bits of each iteration
    int32_t *out;                      // [4] iterations, 0 converged / 1 at the limit
    unsigned long long *guards;
};

constexpr int kSeqWarps = kFloodSlots / 32;
constexpr int kSeqStage = 1024;  // new messages of a level staged in shared memory

__device__ __forceinline__ XP xshfl_idx(const XP &t, int src)
{
    XP r;
    r.m0 = __shfl_sync(0xffffffffu, t.m0, src);
    r.m1 = __shfl_sync(0xffffffffu, t.m1, src);
    r.e0 = __shfl_sync(0xffffffffu, t.e0, src);
    r.e1 = __shfl_sync(0xffffffffu, t.e1, src);
    r.z0 = __shfl_sync(0xffffffffu, t.z0, src);
    r.z1 = __shfl_sync(0xffffffffu, t.z1, src);
    return r;
}

// One warp's edge of a level: the edge, its factor's row, type and
// parameter, and (lane j) the variable at the factor's position j.
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

// The new message of level position li (staged in shared memory, or in S.tmp
// past the stage).
__device__ __forceinline__ float staged(const SeqArgs &S, const float *s_r, int li)
{
    return li < kSeqStage ? s_r[li] : __ldcg(S.tmp + li);
}

// A touched short row (degree <= 8), one thread.  Loaded at the start of the
// level (its entries not written in this level are final for it, and those
// that are come from the stage): the row's entries, phi and the first two
// patches.  Finished after the level's messages are staged: the patches
// applied, the entries multiplied in row order, times phi (the arithmetic of
// the flooding kernels' short rows).
struct ShortPre {
    int v = -1, d = 0, pb = 0, pe = 0;
    float phi = 1.f;
    float r[kFloodSmallMax];
    int2 p0 = make_int2(-1, 0), p1 = make_int2(-1, 0);
};

__device__ __forceinline__ void load_short(ShortPre &P, const SeqArgs &S, const SeqHalfDev &H, int i)
{
    const int4 it = __ldg(H.ds + i);  // {variable, patch begin, patch end, 0}
    P.v = it.x;
    const int lo = __ldg(S.g.vptr + P.v);
    P.d = __ldg(S.g.vptr + P.v + 1) - lo;
    P.phi = __ldg(S.g.phi + P.v);
#pragma unroll
    for (int u = 0; u < kFloodSmallMax; ++u) P.r[u] = u < P.d ? __ldcg(S.a2v_vm + lo + u) : 1.f;
    P.pb = it.y;
    P.pe = it.z;
    if (it.z > it.y) P.p0 = __ldg(H.pt + it.y);
    if (it.z > it.y + 1) P.p1 = __ldg(H.pt + it.y + 1);
}

__device__ __forceinline__ void finish_short(const ShortPre &P, const SeqArgs &S, const SeqHalfDev &H, const float *s_r)
{
    float r[kFloodSmallMax];
#pragma unroll
    for (int u = 0; u < kFloodSmallMax; ++u) r[u] = P.r[u];
    for (int p = P.pb; p < P.pe; ++p) {
        const int2 pc = p == P.pb ? P.p0 : p == P.pb + 1 ? P.p1 : __ldg(H.pt + p);
        const float val = staged(S, s_r, pc.y);
#pragma unroll
        for (int u = 0; u < kFloodSmallMax; ++u)
            if (u == pc.x) r[u] = val;
    }
    XP t = xp_one();
#pragma unroll
    for (int u = 0; u < kFloodSmallMax; ++u)
        if (u < P.d) xmul(t, r[u]);
    xmul(t, P.phi);
    S.F.belief[P.v] = belief_pack(t);
}

// The belief record of a row from its combined product (lane 0 writes).
__device__ __forceinline__ void seq_row_belief(const SeqArgs &S, int v, XP t)
{
    if ((threadIdx.x & 31) != 0) return;
    xmul(t, __ldg(S.g.phi + v));
    S.F.belief[v] = belief_pack(t);
}

// Hub row r whole, by the block (kFloodSlots threads, all calling): thread j
// multiplies slot j's sub-chunks in order, then the butterfly, every node
// kept; the belief from the root.  The same products as the flooding
// kernels' block combine.
__device__ __forceinline__ void seq_hub_full(const SeqArgs &S, int r, XP *s_x)
{
    const int j = threadIdx.x;
    const int4 row = __ldg(S.F.hub_row + r);  // {variable, first agg slot, sub-chunks, 0}
    XP *T = S.tree + (size_t)r * kTreeNodes;
    XP t = xp_one();
    for (int c = j; c < row.z; c += kFloodSlots) t = xcombine(t, ldx<true>(S.F.agg + row.y + c));
    T[kFloodSlots + j] = t;
    for (int k = kFloodSlots / 2; k >= 1; k >>= 1) {
        s_x[j] = t;
        __syncthreads();
        if (j < k) {
            t = xcombine(t, s_x[j + k]);
            T[k + j] = t;
        }
        __syncthreads();
    }
    if (j == 0) {
        xmul(t, __ldg(S.g.phi + row.x));
        S.F.belief[row.x] = belief_pack(t);
    }
}

// A touched sub-chunk, by a whole warp.  Loaded at the start of the level
// (nothing of it depends on the level's new messages): its record, one entry
// per lane, the first two patches, and when the warp finishes the row, the
// row's other products (a medium row's sub-chunks, a hub slot's chain) and
// the hub slot's eight butterfly siblings.  Finished after the level's
// messages are staged: the patches applied, the product in order (every lane
// holds it); a row of one sub-chunk gets its belief; otherwise the product is
// stored and, when this is the row's only touched sub-chunk in the level, the
// row is finished:
//   medium row (2..8 sub-chunks): the flooding kernels' one-thread combine,
//     ((P0 P4)(P2 P6)) ((P1 P5)(P3 P7)) with missing products skipped;
//   hub row: slot s = c mod 256 multiplies its sub-chunks in order again,
//     then the eight butterfly nodes above the slot are combined again with
//     their unchanged siblings (the butterfly combines node (2k, j) with node
//     (2k, j+k) into node (k, j); multiplication commutes, so this is the
//     full butterfly's result bit for bit).
// dk item = {sub-chunk, patch begin, patch end, finish}, finish = 0 (nothing
// more), row << 2 | 2 (medium row), row << 2 | 3 (hub row).
struct SubPre {
    int4 it = make_int4(-1, 0, 0, 0), sc = make_int4(0, 0, 0, 0), row = make_int4(0, 0, 0, 0);
    float x = 1.f;
    int2 p0 = make_int2(-1, 0), p1 = make_int2(-1, 0);
    int fin = 0, r = 0, c = 0, s = 0, nchain = 0, jown = 0;
    XP item, sib;
};

__device__ __forceinline__ void load_sub(SubPre &P, const SeqArgs &S, const SeqHalfDev &H, int i)
{
    const int lane = threadIdx.x & 31;
    P.it = __ldg(H.dk + i);
    P.sc = __ldg(S.F.subs + P.it.x);  // {variable, begin, end, agg slot or -1}
    P.x = P.sc.y + lane < P.sc.z ? __ldcg(S.a2v_vm + P.sc.y + lane) : 1.f;
    if (P.it.z > P.it.y) P.p0 = __ldg(H.pt + P.it.y);
    if (P.it.z > P.it.y + 1) P.p1 = __ldg(H.pt + P.it.y + 1);
    P.fin = P.sc.w < 0 ? 0 : P.it.w & 3;
    P.r = P.it.w >> 2;
    P.item = xp_one();
    P.sib = xp_one();
    if (P.fin == 2) {
        P.row = __ldg(S.F.medium + P.r);  // {variable, first agg slot, sub-chunks, 0}
        P.c = P.sc.w - P.row.y;
        if (lane < P.row.z && lane != P.c) P.item = ldx<true>(S.F.agg + P.row.y + lane);
    } else if (P.fin == 3) {
        P.row = __ldg(S.F.hub_row + P.r);
        P.c = P.sc.w - P.row.y;
        P.s = P.c & (kFloodSlots - 1);
        P.nchain = (P.row.z - P.s + kFloodSlots - 1) / kFloodSlots;
        P.jown = P.c / kFloodSlots;
        if (lane < P.nchain && lane != P.jown) P.item = ldx<true>(S.F.agg + P.row.y + P.s + kFloodSlots * lane);
        if (lane < 8) {
            const int k = (kFloodSlots / 2) >> lane;
            P.sib = ldx<true>(S.tree + (size_t)P.r * kTreeNodes + 2 * k + ((P.s & (2 * k - 1)) ^ k));
        }
    }
}

__device__ __forceinline__ void finish_sub(const SubPre &P, const SeqArgs &S, const SeqHalfDev &H, const float *s_r)
{
    const int lane = threadIdx.x & 31;
    float x = P.x;
    for (int p = P.it.y; p < P.it.z; ++p) {  // warp-uniform
        const int2 pc = p == P.it.y ? P.p0 : p == P.it.y + 1 ? P.p1 : __ldg(H.pt + p);
        if (lane == pc.x) x = staged(S, s_r, pc.y);
    }
    float xs[kFloodSub];
#pragma unroll
    for (int j = 0; j < kFloodSub; ++j) xs[j] = __shfl_sync(0xffffffffu, x, j);
    XP t = xp_one();
    const int len = P.sc.z - P.sc.y;
#pragma unroll
    for (int j = 0; j < kFloodSub; ++j)
        if (j < len) xmul(t, xs[j]);
    if (P.sc.w < 0) {
        seq_row_belief(S, P.sc.x, t);
        return;
    }
    if (lane == 0) S.F.agg[P.sc.w] = t;
    if (P.fin == 2) {
        const int ns = P.row.z;
        const XP mine = lane == P.c ? t : P.item;
        XP Q[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) Q[j] = xshfl_idx(mine, j);
        XP a = Q[0];
        if (ns > 4) a = xcombine(a, Q[4]);
        if (ns > 2) {
            XP u = Q[2];
            if (ns > 6) u = xcombine(u, Q[6]);
            a = xcombine(a, u);
        }
        XP u = Q[1];
        if (ns > 5) u = xcombine(u, Q[5]);
        if (ns > 3) {
            XP u3 = Q[3];
            if (ns > 7) u3 = xcombine(u3, Q[7]);
            u = xcombine(u, u3);
        }
        seq_row_belief(S, P.row.x, xcombine(a, u));
    } else if (P.fin == 3) {
        XP *T = S.tree + (size_t)P.r * kTreeNodes;
        XP cur = xp_one();
        for (int b = 0; b < P.nchain; b += 32) {  // warp-uniform: the slot's sub-chunks, 32 at a time
            const int jj = b + lane;
            XP item = b == 0 ? P.item : xp_one();
            if (b > 0 && jj < P.nchain && jj != P.jown) item = ldx<true>(S.F.agg + P.row.y + P.s + kFloodSlots * jj);
            if (jj == P.jown) item = t;
            const int m = min(32, P.nchain - b);
            for (int j = 0; j < m; ++j) cur = xcombine(cur, xshfl_idx(item, j));
        }
        if (lane == 0) T[kFloodSlots + P.s] = cur;
#pragma unroll
        for (int l = 0; l < 8; ++l) {
            const int k = (kFloodSlots / 2) >> l;
            cur = xcombine(cur, xshfl_idx(P.sib, l));
            if (lane == 0) T[k + (P.s & (k - 1))] = cur;
        }
        seq_row_belief(S, P.row.x, cur);
    }
}

__device__ __forceinline__ void seq_write(const SeqArgs &S, int q, float r)
{
    S.a2v[q] = r;
    S.a2v_vm[__ldg(S.F.vpos + q)] = r;
}


// Every hub row's butterfly nodes and belief from the current sub-chunk
// products, one block per hub row.
__global__ void __launch_bounds__(kFloodSlots) k_seq_trees(const SeqArgs S)
{
    __shared__ XP s_x[kFloodSlots];
    seq_hub_full(S, blockIdx.x, s_x);
}

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
                // the first touched short row of each thread and sub-chunk of
                // each warp, loaded now: step A hides their latency
                const int e0 = __ldg(H.lp + L), e1 = __ldg(H.lp + L + 1);
                const int4 d0 = __ldg(H.dp + L), d1 = __ldg(H.dp + L + 1);
                ShortPre sp;
                if (d0.x + t < d1.x) load_short(sp, S, H, d0.x + t);
                SubPre kp;
                if (d0.y + wp < d1.y) load_sub(kp, S, H, d0.y + wp);  // warp-uniform
                // A: the level's new messages, one warp per edge
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
                // B: the writes, and the touched rows' beliefs from their
                // entries with this level's values patched in
                for (int i = e0 + t; i < e1; i += kFloodSlots) seq_write(S, __ldg(H.le + i), staged(S, s_r, i - e0));
                if (sp.v >= 0) finish_short(sp, S, H, s_r);
                for (int i = d0.x + kFloodSlots + t; i < d1.x; i += kFloodSlots) {
                    ShortPre q;
                    load_short(q, S, H, i);
                    finish_short(q, S, H, s_r);
                }
                if (kp.it.x >= 0) finish_sub(kp, S, H, s_r);  // warp-uniform
                for (int i = d0.y + kSeqWarps + wp; i < d1.y; i += kSeqWarps) {
                    SubPre q;
                    load_sub(q, S, H, i);
                    finish_sub(q, S, H, s_r);
                }
                __syncthreads();
                // C: rows with several touched sub-chunks, whole
                if (d1.z > d0.z || d1.w > d0.w) {  // block-uniform
                    for (int i = d0.z + t; i < d1.z; i += kFloodSlots) belief_medium_item<true>(S.g, S.F, __ldg(H.dm + i));
                    for (int i = d0.w; i < d1.w; ++i) seq_hub_full(S, __ldg(H.dh + i), s_x);
                    __syncthreads();
                }
            }
        }
        // the iteration's residual; stop at the first below tol
        const unsigned bits = __reduce_max_sync(0xffffffffu, __float_as_uint(rmax));
        if (lane == 0) s_res[wp] = bits;
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

// The plan of one level list.  Per level: its edges; every touched short row
// and touched sub-chunk once, with the level's writes into it as patches; a
// row with one touched sub-chunk is finished by that sub-chunk's warp, a row
// with several is listed for the whole recombine.
int build_seq_half(fbp_graph *g, const LevelSet &ls, const std::vector<int32_t> &vpos,
                   const std::vector<int32_t> &sub0, const std::vector<int32_t> &row_of, SeqHalf &out)
{
    const HostCSR &h = g->h;
    const int32_t nl = ls.lp.empty() ? 0 : (int32_t)ls.lp.size() - 1;
    std::vector<int32_t> lp(nl + 1), dm, dh;
    std::vector<int4> dp(nl + 1), ds, dk;
    std::vector<int2> pt;
    struct Touch {
        int32_t v, c, pos, li;  // variable, sub-chunk in its row (-1: a short row), position, index in the level
    };
    std::vector<Touch> T;
    int32_t widest = 0;
    for (int32_t L = 0; L < nl; ++L) {
        lp[L] = (int32_t)ls.lp[L];
        dp[L] = make_int4((int)ds.size(), (int)dk.size(), (int)dm.size(), (int)dh.size());
        const int64_t e0 = ls.lp[L], e1 = ls.lp[L + 1];
        widest = std::max(widest, (int32_t)(e1 - e0));
        T.clear();
        for (int64_t i = e0; i < e1; ++i) {
            const int32_t q = ls.le[i], v = h.fvars[q];
            const int32_t lo = h.vptr[v], d = h.vptr[v + 1] - lo, k = vpos[q] - lo;
            if (d <= kFloodSmallMax) T.push_back({v, -1, k, (int32_t)(i - e0)});
            else T.push_back({v, k / kFloodSub, k % kFloodSub, (int32_t)(i - e0)});
        }
        std::sort(T.begin(), T.end(), [](const Touch &a, const Touch &b) {
            return a.v != b.v ? a.v < b.v : a.c != b.c ? a.c < b.c : a.li < b.li;
        });
        for (size_t a = 0; a < T.size();) {
            size_t b = a;
            while (b < T.size() && T[b].v == T[a].v) ++b;
            const int32_t v = T[a].v;
            if (T[a].c < 0) {  // a short row
                const int pb = (int)pt.size();
                for (size_t x = a; x < b; ++x) pt.push_back(make_int2(T[x].pos, T[x].li));
                ds.push_back(make_int4(v, pb, (int)pt.size(), 0));
            } else {
                int n_subs = 0;
                for (size_t x = a; x < b; ++x) n_subs += x == a || T[x].c != T[x - 1].c;
                const int32_t d = h.vptr[v + 1] - h.vptr[v], ns = (d + kFloodSub - 1) / kFloodSub;
                int fin = 0;
                if (ns > 1 && n_subs == 1) fin = row_of[v] >= 0 ? (row_of[v] << 2 | 2) : ((-2 - row_of[v]) << 2 | 3);
                if (ns > 1 && n_subs > 1) (row_of[v] >= 0 ? dm : dh).push_back(row_of[v] >= 0 ? row_of[v] : -2 - row_of[v]);
                for (size_t x = a; x < b;) {
                    size_t y = x;
                    const int pb = (int)pt.size();
                    while (y < b && T[y].c == T[x].c) pt.push_back(make_int2(T[y].pos, T[y].li)), ++y;
                    dk.push_back(make_int4(sub0[v] + T[x].c, pb, (int)pt.size(), fin));
                    x = y;
                }
            }
            a = b;
        }
    }
    lp[nl] = nl > 0 ? (int32_t)ls.lp[nl] : 0;
    dp[nl] = make_int4((int)ds.size(), (int)dk.size(), (int)dm.size(), (int)dh.size());
    out.n_levels = nl;
    out.max_level = widest;
    int rc = upload(g, &out.lp, lp.data(), lp.size());
    if (!rc) rc = upload(g, &out.le, ls.le.data(), ls.le.size());
    if (!rc) rc = upload(g, &out.dp, dp.data(), dp.size());
    if (!rc) rc = upload(g, &out.ds, ds.data(), ds.size());
    if (!rc) rc = upload(g, &out.dk, dk.data(), dk.size());
    if (!rc) rc = upload(g, &out.dm, dm.data(), dm.size());
    if (!rc) rc = upload(g, &out.dh, dh.data(), dh.size());
    if (!rc) rc = upload(g, &out.pt, pt.data(), pt.size());
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
    int rc = FBP_OK;
    for (size_t k = 0; k < g->halves.size() && !rc; ++k) {
        rc = build_seq_half(g, g->halves[k], vpos, sub0, row_of, g->seq[k]);
        wide = std::max<int64_t>(wide, g->seq[k].max_level);
    }
    if (!rc && wide > kSeqStage && !(rc = dalloc_n(g, &g->seq_tmp, (size_t)wide))) g->seq_tmp_cap = wide;
    if (!rc) rc = dalloc_n(g, &g->seq_tree, std::max<size_t>(g->flood_hub_h.size(), 1) * kTreeNodes);
    if (rc) free_seq(g);
    return rc;
}

SeqHalfDev half_dev(const SeqHalf &s)
{
    return SeqHalfDev{s.n_levels, s.lp, s.le, s.dp, s.ds, s.dk, s.dm, s.dh, s.pt};
}

}  // namespace

void free_seq(fbp_graph *g)
{
    for (auto &s : g->seq) {
        for (void *p : {(void *)s.lp, (void *)s.le, (void *)s.dp, (void *)s.ds, (void *)s.dk, (void *)s.dm, (void *)s.dh,
                        (void *)s.pt})
            dfree(g, p);
    }
    g->seq.clear();
    dfree(g, g->seq_tmp);
    g->seq_tmp = nullptr;
    g->seq_tmp_cap = 0;
    dfree(g, g->seq_tree);
    g->seq_tree = nullptr;
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
    // the beliefs of the current messages (one flooding phase 1), then every
    // hub row's butterfly nodes from the same sub-chunk products
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
    S.tree = g->seq_tree;
    S.half[0] = half_dev(g->seq[0]);
    S.half[1] = g->seq.size() > 1 ? half_dev(g->seq[1]) : SeqHalfDev{};
    S.n_halves = (int32_t)g->seq.size();
    S.max_iters = max_iters;
    S.tol = (float)tol;
    S.res = g->d_res_it;
    S.out = g->d_out;
    S.guards = g->d_guards;
    const int n_hubs = (int)g->flood_hub_h.size();
    if (n_hubs > 0) k_seq_trees<<<n_hubs, kFloodSlots, 0, g->stream>>>(S);
    k_seq_belief<<<1, kFloodSlots, 0, g->stream>>>(S);
    SEQ_TRY(cudaGetLastError());
    g->stats.kernel_launches += 2 + (n_hubs > 0) + (flood_launches(g->d, g->flood) > 3 ? 2 : 1);
    if ((rc = engine_check(g))) return rc;
    const int32_t it = g->h_out[0];
    const int status = g->h_out[1] == 0 ? FBP_OK : FBP_NOT_CONVERGED;
    int64_t per_iter = 0;
    for (auto &ls : g->halves) per_iter += (int64_t)ls.le.size();
    g->stats.updates += (int64_t)it * per_iter;
    return finish_run(g, it, residual_at(g, it), status, iters_out, residual_out);
}

}  // namespace fbp
