// Flooding (PARALL) iteration kernels (sm_103a), for graphs of any degree
// distribution (BINGO-shaped derivation graphs have hub variables with 1e5
// incident factors next to millions of degree-2 variables).
//
// Phase 1, Eq. (1): mu_{v->a} = phi_v * prod_{b != a} mu_{b->v}.  Instead of
// prefix/suffix products (scans), each variable row is reduced once to its
// total product and every entry's message is total / own factor.  This is
// exact in the algebra of the messages as long as (i) exact zeros (hard
// messages) are counted rather than multiplied in, and (ii) the product never
// underflows: each of the two entries is kept as a mantissa in [1/2, 1) and an
// integer exponent.  Rounding is one multiply per factor (tree-shaped across
// lanes and blocks for long rows) and one divide per entry.
//   rows of degree 1 or 2     one thread per row (lean kernel)
//   rows of degree 3..8       one thread per row; prefix/suffix products in
//                             registers (multiply-only, as in the oracle)
//   rows of degree <= 256     one warp per row
//   longer rows (hubs)        chunks of kFloodHubChunk entries, one block each; a
//                             pre-pass writes the partial product of each
//                             256-entry sub-chunk
// The row total of every row longer than 8 entries is grouped one way only,
// whichever kernel carries the row: the row is cut into 256-entry sub-chunks;
// lane l of a warp multiplies entries l, l+32, ..., l+224 of a sub-chunk in
// that order and the 32 lane products are combined by an xor butterfly; the
// sub-chunk products are then combined the same way (lane j takes sub-chunks
// j, j+32, ... in order, then the butterfly).  A row of at most 256 entries is
// one sub-chunk, so the warp-per-row path and the chunked path compute the
// same bits, and the split thresholds (FBP_OPT_FLOOD_HUB_MIN, _CHUNK) only
// move work between kernels.  Every multiply rounds the exact product once
// (the mantissa/exponent form never goes subnormal), so only this grouping
// decides the result.
// Phase 2, the closed-form local-structure messages: one lane per message,
// whole factors per warp, the factor's other messages by warp shuffle;
// factors wider than a warp one thread per edge.
#include "fbp_msg.cuh"
#include "fbp_flood.h"

namespace fbp {

namespace {

__device__ __forceinline__ XP xp_one() { return XP{1.f, 1.f, 0, 0, 0, 0}; }

// In a batch, rows and factors of graphs that have stopped are skipped.
__device__ __forceinline__ bool var_frozen(const FloodPlanDev &F, int v)
{
    return F.batch.n_graphs > 0 && __ldcg(F.batch.done + __ldg(F.vgraph + v)) != 0;
}

// Multiply entry (m, e, z) by x in [0, 1]: exact zeros are counted; the
// mantissa is renormalised into [1/2, 1) only when the product falls below
// 2^-60, so the common case is one multiply and one compare.
__device__ __forceinline__ void xmul1(float &m, int &e, int &z, float x)
{
    if (x == 0.f) {
        ++z;
        return;
    }
    const float p = m * x;
    if (p < 0x1p-60f) {
        int em, ex, pe;
        const float mm = frexpf(m, &em), mx = frexpf(x, &ex);
        m = frexpf(mm * mx, &pe);
        e += em + ex + pe;
        return;
    }
    m = p;
}

__device__ __forceinline__ void xmul(XP &t, float rho)
{
    const P2 x = dec(rho);
    xmul1(t.m0, t.e0, t.z0, x.m0);
    xmul1(t.m1, t.e1, t.z1, x.m1);
}

__device__ __forceinline__ XP xcombine(const XP &a, const XP &b)
{
    XP r;
    float p0 = a.m0 * b.m0, p1 = a.m1 * b.m1;
    r.e0 = a.e0 + b.e0;
    r.e1 = a.e1 + b.e1;
    int k0, k1;
    p0 = frexpf(p0, &k0);
    p1 = frexpf(p1, &k1);
    r.m0 = p0;
    r.m1 = p1;
    r.e0 += k0;
    r.e1 += k1;
    r.z0 = a.z0 + b.z0;
    r.z1 = a.z1 + b.z1;
    return r;
}

__device__ __forceinline__ XP xshfl_xor(const XP &t, int o)
{
    XP r;
    r.m0 = __shfl_xor_sync(0xffffffffu, t.m0, o);
    r.m1 = __shfl_xor_sync(0xffffffffu, t.m1, o);
    r.e0 = __shfl_xor_sync(0xffffffffu, t.e0, o);
    r.e1 = __shfl_xor_sync(0xffffffffu, t.e1, o);
    r.z0 = __shfl_xor_sync(0xffffffffu, t.z0, o);
    r.z1 = __shfl_xor_sync(0xffffffffu, t.z1, o);
    return r;
}

__device__ __forceinline__ XP warp_product(XP t)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = xcombine(t, xshfl_xor(t, o));
    return t;
}

// Block-wide product (all threads get the result).  blockDim.x <= 1024.
__device__ __forceinline__ XP block_product(XP t)
{
    __shared__ XP s_x[32];
    t = warp_product(t);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) s_x[w] = t;
    __syncthreads();
    XP u = lane < nw ? s_x[lane] : xp_one();
    u = warp_product(u);
    return u;
}

// frexp of an entry that is nonzero, or of 1 for an entry counted as zero.
__device__ __forceinline__ float fx(float x, int &e)
{
    return frexpf(x == 0.f ? 1.f : x, &e);
}

// v->a message of an entry with factor rho_k, from the row total t and phi:
// phi * t / x_k, encoded; zero mass -> uniform.  The ratio of the two entries
// is (t0 f0 x1) / (t1 f1 x0), formed from mantissas in [1/2, 1) and an exponent
// difference, so nothing underflows before the final encoding.
__device__ __forceinline__ float excl_msg(const XP &t, float phi, float rho_k)
{
    const P2 f = dec(phi), x = dec(rho_k);
    const int z0 = t.z0 - (x.m0 == 0.f) + (f.m0 == 0.f);
    const int z1 = t.z1 - (x.m1 == 0.f) + (f.m1 == 0.f);
    if (z0 > 0 && z1 > 0) return 1.f;  // zero mass: uniform
    if (z0 > 0) return 0.f;            // hard (0, 1)
    if (z1 > 0) return -0.f;           // hard (1, 0)
    const float f0 = f.m0 == 0.f ? 1.f : f.m0, f1 = f.m1 == 0.f ? 1.f : f.m1;
    const float x0 = x.m0 == 0.f ? 1.f : x.m0, x1 = x.m1 == 0.f ? 1.f : x.m1;
    float n0, n1;
    int de;
    if (fminf(fminf(f0, f1), fminf(x0, x1)) >= 0x1p-30f) {
        // t.m >= 2^-60 and the rest >= 2^-30: both products stay normal
        n0 = t.m0 * f0 * x1;
        n1 = t.m1 * f1 * x0;
        de = t.e0 - t.e1;
    } else {
        int ef0, ef1, ex0, ex1;
        n0 = t.m0 * fx(f0, ef0) * fx(x1, ex1);
        n1 = t.m1 * fx(f1, ef1) * fx(x0, ex0);
        de = (t.e0 + ef0 + ex1) - (t.e1 + ef1 + ex0);
    }
    de = max(-400, min(400, de));
    const float r = ldexpf(__fdiv_rn(n0, n1), de);
    if (r <= 1.f) return r;            // m1 is the larger entry
    return -__frcp_rn(r);              // m0 is the larger entry
}

// ----------------------------------------------------------------------------
// Phase 1
// ----------------------------------------------------------------------------
// Product of one 256-entry sub-chunk [b, end) of a row, by one warp, in the
// canonical grouping (all lanes get it).  Entries past `end` multiply by 1,
// which is exact.
__device__ __forceinline__ XP sub_chunk_product(const DevGraph &g, const float *__restrict__ a2v, int b, int end,
                                                int lane, int *e, float *r)
{
    const int ns = (end - b + 31) >> 5;  // slots in use (warp-uniform); the others would multiply by 1
#pragma unroll
    for (int u = 0; u < kFloodSub / 32; ++u)
        e[u] = u < ns && b + lane + 32 * u < end ? __ldg(g.vedge + b + lane + 32 * u) : -1;
#pragma unroll
    for (int u = 0; u < kFloodSub / 32; ++u) r[u] = e[u] >= 0 ? __ldg(a2v + e[u]) : 1.f;
    XP t = xp_one();
#pragma unroll
    for (int u = 0; u < kFloodSub / 32; ++u)
        if (u < ns) xmul(t, r[u]);
    return warp_product(t);
}

// Partial products of the 256-entry sub-chunks of one chunk of a hub row; the
// chunk's warps take its sub-chunks in turn.
__global__ void __launch_bounds__(256) k_hub_partials(const DevGraph g, FloodPlanDev F,
                                                      const float *__restrict__ a2v)
{
    if (*(volatile const int *)F.done) return;
    const int c = blockIdx.x;
    const int4 ch = __ldg(F.hub + c);  // {var, begin, end, first sub-chunk of this chunk}
    if (var_frozen(F, ch.x)) return;   // block-uniform
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int nsub = (ch.z - ch.y + kFloodSub - 1) / kFloodSub;
    for (int s = threadIdx.x >> 5; s < nsub; s += nw) {
        int e[kFloodSub / 32];
        float r[kFloodSub / 32];
        const int b = ch.y + s * kFloodSub;
        const XP t = sub_chunk_product(g, a2v, b, min(ch.z, b + kFloodSub), lane, e, r);
        if (lane == 0) F.agg[ch.w + s] = t;
    }
}

// Variables of degree 1 and 2 (most of a derivation graph: every rule's
// derivation variable has degree 2): one thread each, few registers.
__global__ void __launch_bounds__(256) k_v2a_lean(const DevGraph g, const FloodPlanDev F,
                                                  const float *__restrict__ a2v, float *__restrict__ v2a)
{
    if (*(volatile const int *)F.done) return;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= g.nv || var_frozen(F, v)) return;
    const int lo = __ldg(g.vptr + v), d = __ldg(g.vptr + v + 1) - lo;
    if (d == 0 || d > 2) return;
    const P2 f = dec(__ldg(g.phi + v));
    bool gd = false;
    if (d == 1) {
        v2a[__ldg(g.vedge + lo)] = enc_fast(f, gd);
        return;
    }
    const int e0 = __ldg(g.vedge + lo), e1 = __ldg(g.vedge + lo + 1);
    const P2 x0 = dec(__ldg(a2v + e0)), x1 = dec(__ldg(a2v + e1));
    v2a[e0] = enc_fast(mul(f, x1), gd);  // each message is phi times the other one
    v2a[e1] = enc_fast(mul(f, x0), gd);
}

// The other rows, from host-built lists: degree 3..8 one thread each (prefix
// and suffix products in registers), 9..256 one warp each (row total and
// division), longer rows in chunks (the chunk partials combined first).
__global__ void __launch_bounds__(256) k_v2a_rest(const DevGraph g, FloodPlanDev F,
                                                  const float *__restrict__ a2v, float *__restrict__ v2a)
{
    if (*(volatile const int *)F.done) return;
    const int b = blockIdx.x;
    if (b < F.nb_small) {
        const int i = b * blockDim.x + threadIdx.x;
        if (i >= F.n_small) return;
        const int v = __ldg(F.small + i);
        if (var_frozen(F, v)) return;
        const int lo = __ldg(g.vptr + v), d = __ldg(g.vptr + v + 1) - lo;
        const P2 f = dec(__ldg(g.phi + v));
        bool gd = false;
        int e[kFloodSmallMax];
        P2 x[kFloodSmallMax], pre[kFloodSmallMax];
#pragma unroll
        for (int u = 0; u < kFloodSmallMax; ++u) e[u] = u < d ? __ldg(g.vedge + lo + u) : 0;
#pragma unroll
        for (int u = 0; u < kFloodSmallMax; ++u) x[u] = dec(u < d ? __ldg(a2v + e[u]) : 1.f);
        P2 acc = f;
#pragma unroll
        for (int u = 0; u < kFloodSmallMax; ++u) {
            if (u < d) {  // the list is sorted by degree, so d is nearly uniform in a warp
                pre[u] = acc;
                acc = mul(acc, x[u]);
                resc(acc);
            }
        }
        P2 suf{1.f, 1.f};
#pragma unroll
        for (int u = kFloodSmallMax - 1; u >= 0; --u) {
            if (u < d) {
                P2 m = mul(pre[u], suf);
                resc(m);
                v2a[e[u]] = enc_fast(m, gd);
                suf = mul(suf, x[u]);
                resc(suf);
            }
        }
        return;
    }
    const int bm = b - F.nb_small;
    if (bm < F.nb_medium) {
        // one warp per variable of degree in (kFloodSmallMax, kFloodMediumMax]:
        // the row is a single sub-chunk
        const int w = bm * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
        if (w >= F.n_medium) return;
        const int v = __ldg(F.medium + w);
        if (var_frozen(F, v)) return;
        const int lo = __ldg(g.vptr + v), hi = __ldg(g.vptr + v + 1);
        int e[kFloodSub / 32];
        float r[kFloodSub / 32];
        const XP t = sub_chunk_product(g, a2v, lo, hi, lane, e, r);
        const float phi = __ldg(g.phi + v);
#pragma unroll
        for (int u = 0; u < kFloodSub / 32; ++u)
            if (e[u] >= 0) v2a[e[u]] = excl_msg(t, phi, r[u]);
        return;
    }
    // hub chunk: combine the row's sub-chunk partials (canonical grouping),
    // then every entry of this chunk
    const int c = bm - F.nb_medium;
    const int4 ch = __ldg(F.hub + c);
    if (var_frozen(F, ch.x)) return;  // block-uniform
    const int2 rs = __ldg(F.hub_row + c);  // {first sub-chunk of the row, sub-chunks of the row}
    __shared__ XP s_tot;
    if (threadIdx.x < 32) {
        XP t = xp_one();
        for (int j = threadIdx.x; j < rs.y; j += 32) t = xcombine(t, F.agg[rs.x + j]);
        t = warp_product(t);
        if (threadIdx.x == 0) s_tot = t;
    }
    __syncthreads();
    const XP t = s_tot;
    const float phi = __ldg(g.phi + ch.x);
    for (int k0 = ch.y + threadIdx.x; k0 < ch.z; k0 += 4 * blockDim.x) {
        int e[4];
        float r[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) e[u] = k0 + u * blockDim.x < ch.z ? __ldg(g.vedge + k0 + u * blockDim.x) : -1;
#pragma unroll
        for (int u = 0; u < 4; ++u) r[u] = e[u] >= 0 ? __ldg(a2v + e[u]) : 1.f;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (e[u] >= 0) v2a[e[u]] = excl_msg(t, phi, r[u]);
    }
}

// ----------------------------------------------------------------------------
// Phase 2
// ----------------------------------------------------------------------------
// Per-graph residual of a batch: one atomic per graph present in the warp.
__device__ __forceinline__ void batch_residual(const FloodPlanDev &F, int graph, float d)
{
    const unsigned grp = __match_any_sync(0xffffffffu, graph);
    const unsigned bits = __reduce_max_sync(grp, __float_as_uint(d));
    if (graph >= 0 && (threadIdx.x & 31) == __ffs(grp) - 1 && bits) max_bits(F.batch.res + graph, bits);
}

// One lane per message: each warp holds whole factors (consecutive in the
// factor-major order, so its edges are one contiguous range and every load
// and the store are coalesced).  A lane reads its own incoming v->a message;
// the factor's other messages come from the neighbouring lanes by shuffle, in
// premise order (the order of a2v_unified, so the arithmetic is the level
// engine's), over a trip count that is uniform in the warp, so that factors of
// different types and fan-ins in one warp run one instruction stream.  A
// factor of at most 32 variables has Ps <= 2^31, so the products need no
// rescaling here.  The a->v messages are written in place: phase 2 reads only
// v->a messages.
__global__ void __launch_bounds__(256) k_a2v_lanes(const DevGraph g, const FloodPlanDev F,
                                                   const float *__restrict__ v2a, float *__restrict__ a2v, IterCtl ctl)
{
    if (*(volatile const int *)F.done) return;
    __shared__ float s_x[256];  // the lanes' incoming messages (generic factors read them here)
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    float d = 0.f;
    unsigned long long ng = 0;
    int graph = -1;
    if (w < F.n_warps) {  // warp-uniform
        const int4 wr = __ldg(F.warps + w);  // {first edge, end edge, first factor, end factor}
        const int e = wr.x + lane;
        const bool valid = e < wr.y;
        int lo = wr.x, n = 1, type = 0, a = 0;
        float p = 0.f, x = 1.f, old = 1.f;
        bool frozen = false;
        if (valid) {
            a = __ldg(g.efac + e);
            lo = __ldg(g.fptr + a);
            n = __ldg(g.fptr + a + 1) - lo;
            type = __ldg(g.ftype + a);
            p = __ldg(g.fparam + a);
            x = __ldg(v2a + e);
            old = a2v[e];
            if (F.batch.n_graphs > 0) {
                graph = __ldg(F.fgraph + a);
                frozen = __ldcg(F.batch.done + graph) != 0;
            }
        }
        const int first = lo - wr.x, i = e - lo, y = n - 1;
        const int span = __reduce_max_sync(0xffffffffu, valid ? y : 0);
        Acc5 A;
        for (int j = 0; j < span; ++j) {
            const float r = __shfl_sync(0xffffffffu, x, (first + j) & 31);
            if (j < y && j != i) {
                const P2 m = dec(r);
                const float s = m.m0 + m.m1;
                A.D = fmaf(A.D, s, A.P1 * m.m0);
                A.D0 = fmaf(A.D0, s, A.P0 * m.m1);
                A.P1 *= m.m1;
                A.P0 *= m.m0;
                A.Ps *= s;
            }
        }
        const float ry = __shfl_sync(0xffffffffu, x, (first + y) & 31);
        s_x[threadIdx.x] = x;
        __syncwarp();
        const bool write = valid && !frozen && (!F.elevel || __ldg(F.elevel + e) == F.level);
        if (write) {
            const float *wx = s_x + (threadIdx.x & ~31) + first;
            const P2 mu = type == kTypeTERMS ? a2v_terms(g, a, n, i, [&](int j) { return dec(wx[j]); })
                                             : a2v_finish(type, p, i == y, A, dec(ry));
            bool gd = false;
            const float r = enc_fast(mu, gd);
            ng += gd;
            d = delta_p1_fast(r, old);
            a2v[e] = r;
            if (F.dres) F.dres[e] = d;
        }
    }
    if (ng) atomicAdd(ctl.guards, ng);
    if (F.batch.n_graphs > 0) {
        batch_residual(F, graph, d);
        return;
    }
    const float bm = block_max(d);
    if (threadIdx.x == 0 && bm > 0.f) max_bits(ctl.res + (blockIdx.x % kResSlots), __float_as_uint(bm));
}

// Factors wider than a warp: one thread per edge, the closed form over the
// factor's v->a messages read from memory.
__global__ void __launch_bounds__(256) k_a2v_wide(const DevGraph g, const FloodPlanDev F,
                                                  const float *__restrict__ v2a, float *__restrict__ a2v, IterCtl ctl)
{
    if (*(volatile const int *)F.done) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    float d = 0.f;
    unsigned long long ng = 0;
    int graph = -1;
    if (k < F.n_wide) {
        const int e = __ldg(F.wide + k);
        const int a = __ldg(g.efac + e);
        const int lo = __ldg(g.fptr + a), n = __ldg(g.fptr + a + 1) - lo;
        bool frozen = false;
        if (F.batch.n_graphs > 0) {
            graph = __ldg(F.fgraph + a);
            frozen = __ldcg(F.batch.done + graph) != 0;
        }
        if (!frozen && (!F.elevel || __ldg(F.elevel + e) == F.level)) {
            const P2 mu = a2v_unified(__ldg(g.ftype + a), __ldg(g.fparam + a), n, e - lo,
                                      [&](int j) { return dec(__ldg(v2a + lo + j)); });
            bool gd = false;
            const float r = enc_fast(mu, gd);
            ng += gd;
            d = delta_p1_fast(r, a2v[e]);
            a2v[e] = r;
            if (F.dres) F.dres[e] = d;
        }
    }
    if (ng) atomicAdd(ctl.guards, ng);
    if (F.batch.n_graphs > 0) {
        batch_residual(F, graph, d);
        return;
    }
    const float bm = block_max(d);
    if (threadIdx.x == 0 && bm > 0.f) max_bits(ctl.res + (blockIdx.x % kResSlots), __float_as_uint(bm));
}

// End of an iteration of a batch: per-graph bookkeeping as in the persistent
// engine; the run is done when no graph is running.  The iteration number is
// the device's own count (ctl[1] + 1), so a captured chunk of iterations can
// be replayed.
__global__ void k_flood_batch_check(BatchCtl B, int *ctl)
{
    if (*(volatile int *)ctl) return;
    const int it = ctl[1] + 1;
    __shared__ int s_active;
    if (threadIdx.x == 0) s_active = 0;
    __syncthreads();
    int act = 0;
    for (int gi = threadIdx.x; gi < B.n_graphs; gi += blockDim.x) {
        if (B.done[gi]) continue;
        const unsigned r = B.res[gi];
        B.res[gi] = 0u;
        B.last_res[gi] = r;
        B.iters[gi] = it;
        if (__uint_as_float(r) < B.tol[gi]) B.done[gi] = 1;
        else if (it >= B.max_iters[gi]) B.done[gi] = 2;
        else ++act;
    }
    act = __reduce_add_sync(0xffffffffu, act);
    if ((threadIdx.x & 31) == 0 && act) atomicAdd(&s_active, act);
    __syncthreads();
    if (threadIdx.x == 0) {
        ctl[1] = it;
        if (s_active == 0 || it >= ctl[3]) ctl[0] = 1;
    }
}

// End of an iteration: the residual of iteration it = ctl[1] + 1 is the max
// over the slots; the slots are cleared for the next iteration; the run is
// marked done (ctl[0] = 1) at the first iteration below tol, or (ctl[0] = 2)
// at the iteration limit ctl[3].  Later iterations see the flag and return at
// once.
__global__ void k_flood_check(unsigned *slots, unsigned *hist, float tol, int *ctl)
{
    if (*(volatile int *)ctl) return;
    const int it = ctl[1] + 1;
    const unsigned v = threadIdx.x < kResSlots ? slots[threadIdx.x] : 0u;
    const unsigned m = __reduce_max_sync(0xffffffffu, v);
    __shared__ unsigned s_m[kResSlots / 32];
    if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < kResSlots) slots[threadIdx.x] = 0u;
    if (threadIdx.x == 0) {
        unsigned r = 0;
        for (int i = 0; i < kResSlots / 32; ++i) r = max(r, s_m[i]);
        hist[it - 1] = r;
        ctl[1] = it;
        if (__uint_as_float(r) < tol) ctl[0] = 1;
        else if (it >= ctl[3]) ctl[0] = 2;
    }
}

}  // namespace

void flood_iteration(const DevGraph &g, const FloodPlanDev &F, float *a2v, float *v2a, IterCtl ctl, float tol,
                     unsigned *hist, int *done, cudaStream_t s)
{
    FloodPlanDev P = F;
    P.done = done;
    if (g.nv > 0) k_v2a_lean<<<(g.nv + 255) / 256, 256, 0, s>>>(g, P, a2v, v2a);
    if (P.n_hub > 0) k_hub_partials<<<P.n_hub, 256, 0, s>>>(g, P, a2v);
    const int nb = P.nb_small + P.nb_medium + P.n_hub;
    if (nb > 0) k_v2a_rest<<<nb, 256, 0, s>>>(g, P, a2v, v2a);
    if (P.n_warps > 0) k_a2v_lanes<<<(P.n_warps + 7) / 8, 256, 0, s>>>(g, P, v2a, a2v, ctl);
    if (P.n_wide > 0) k_a2v_wide<<<(P.n_wide + 255) / 256, 256, 0, s>>>(g, P, v2a, a2v, ctl);
    if (P.batch.n_graphs > 0) k_flood_batch_check<<<1, 1024, 0, s>>>(P.batch, done);
    else k_flood_check<<<1, kResSlots, 0, s>>>(ctl.res, hist, tol, done);
}

void flood_level(const DevGraph &g, const FloodPlanDev &F, float *a2v, float *v2a, IterCtl ctl, int *done,
                 cudaStream_t s)
{
    FloodPlanDev P = F;
    P.done = done;
    if (g.nv > 0) k_v2a_lean<<<(g.nv + 255) / 256, 256, 0, s>>>(g, P, a2v, v2a);
    if (P.n_hub > 0) k_hub_partials<<<P.n_hub, 256, 0, s>>>(g, P, a2v);
    const int nb = P.nb_small + P.nb_medium + P.n_hub;
    if (nb > 0) k_v2a_rest<<<nb, 256, 0, s>>>(g, P, a2v, v2a);
    if (P.n_warps > 0) k_a2v_lanes<<<(P.n_warps + 7) / 8, 256, 0, s>>>(g, P, v2a, a2v, ctl);
    if (P.n_wide > 0) k_a2v_wide<<<(P.n_wide + 255) / 256, 256, 0, s>>>(g, P, v2a, a2v, ctl);
}

void flood_check(IterCtl ctl, float tol, unsigned *hist, int *done, cudaStream_t s)
{
    k_flood_check<<<1, kResSlots, 0, s>>>(ctl.res, hist, tol, done);
}

cudaError_t flood_capture(const DevGraph &g, const FloodPlanDev &F, float *a2v, float *v2a, IterCtl ctl, float tol,
                          unsigned *hist, int *done, int iters, cudaGraphExec_t *exec)
{
    cudaStream_t cap = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int k = 0; k < iters; ++k) flood_iteration(g, F, a2v, v2a, ctl, tol, hist, done, cap);
        const cudaError_t launch = cudaGetLastError();
        e = cudaStreamEndCapture(cap, &graph);
        if (e == cudaSuccess && launch != cudaSuccess) e = launch;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    return e;
}

int flood_launches(const DevGraph &g, const FloodPlanDev &F)
{
    return (g.nv > 0) + (F.n_hub > 0) + (F.nb_small + F.nb_medium + F.n_hub > 0) + (F.n_warps > 0) +
           (F.n_wide > 0) + 1;
}

}  // namespace fbp
