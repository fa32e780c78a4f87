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
//                             pre-pass writes each chunk's partial product
// Phase 2, the closed-form local-structure messages: one thread per factor,
// the block's factor rows staged through shared memory so that the v->a reads
// and the a->v read-modify-write are coalesced.
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
__global__ void __launch_bounds__(256) k_hub_partials(const DevGraph g, FloodPlanDev F,
                                                      const float *__restrict__ a2v)
{
    if (*(volatile const int *)F.done) return;
    const int c = blockIdx.x;
    const int4 ch = __ldg(F.hub + c);  // {var, begin, end, first chunk of the row}
    if (var_frozen(F, ch.x)) return;   // block-uniform
    XP t = xp_one();
    for (int k0 = ch.y + threadIdx.x; k0 < ch.z; k0 += 4 * blockDim.x) {
        int e[4];
        float r[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) e[u] = k0 + u * blockDim.x < ch.z ? __ldg(g.vedge + k0 + u * blockDim.x) : -1;
#pragma unroll
        for (int u = 0; u < 4; ++u) r[u] = e[u] >= 0 ? __ldg(a2v + e[u]) : 1.f;
#pragma unroll
        for (int u = 0; u < 4; ++u) xmul(t, r[u]);
    }
    t = block_product(t);
    if (threadIdx.x == 0) F.agg[c] = t;
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
            pre[u] = acc;
            acc = mul(acc, x[u]);
            resc(acc);
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
        // one warp per variable of degree in (kFloodSmallMax, kFloodMediumMax]
        const int w = bm * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
        if (w >= F.n_medium) return;
        const int v = __ldg(F.medium + w);
        if (var_frozen(F, v)) return;
        const int lo = __ldg(g.vptr + v), hi = __ldg(g.vptr + v + 1);
        // at most kFloodMediumMax / 32 = 8 entries per lane, all loads issued first
        int e[kFloodMediumMax / 32];
        float r[kFloodMediumMax / 32];
#pragma unroll
        for (int u = 0; u < kFloodMediumMax / 32; ++u) e[u] = lo + lane + 32 * u < hi ? __ldg(g.vedge + lo + lane + 32 * u) : -1;
#pragma unroll
        for (int u = 0; u < kFloodMediumMax / 32; ++u) r[u] = e[u] >= 0 ? __ldg(a2v + e[u]) : 1.f;
        XP t = xp_one();
#pragma unroll
        for (int u = 0; u < kFloodMediumMax / 32; ++u) xmul(t, r[u]);
        t = warp_product(t);
        const float phi = __ldg(g.phi + v);
#pragma unroll
        for (int u = 0; u < kFloodMediumMax / 32; ++u)
            if (e[u] >= 0) v2a[e[u]] = excl_msg(t, phi, r[u]);
        return;
    }
    // hub chunk: combine the row's chunk partials, then every entry of this chunk
    const int c = bm - F.nb_medium;
    const int4 ch = __ldg(F.hub + c);
    if (var_frozen(F, ch.x)) return;  // block-uniform
    const int c0 = ch.w, nc = __ldg(F.hub_nchunks + c);
    __shared__ XP s_tot;
    if (threadIdx.x < 32) {
        XP t = xp_one();
        for (int j = threadIdx.x; j < nc; j += 32) t = xcombine(t, F.agg[c0 + j]);
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
// Accumulators of the closed forms over a run of premises (fbp_msg.cuh):
// P1, P0, Ps and the first-false sums D, D0.  Runs concatenate exactly:
//   P(A.B) = P(A) P(B),  D(A.B) = D(A) Ps(B) + P1(A) D(B),
//   D0(A.B) = D0(A) Ps(B) + P0(A) D0(B),
// which gives every target's "all premises but one" accumulators from one
// forward (prefix) and one backward (suffix) pass: O(n) per factor.
struct Acc {
    float P1, P0, Ps, D, D0;
};

__device__ __forceinline__ Acc acc_one() { return Acc{1.f, 1.f, 1.f, 0.f, 0.f}; }

__device__ __forceinline__ Acc acc_append(const Acc &a, P2 m)  // A . {m}
{
    const float s = m.m0 + m.m1;
    return Acc{a.P1 * m.m1, a.P0 * m.m0, a.Ps * s, fmaf(a.D, s, a.P1 * m.m0), fmaf(a.D0, s, a.P0 * m.m1)};
}

__device__ __forceinline__ Acc acc_prepend(P2 m, const Acc &b)  // {m} . B
{
    const float s = m.m0 + m.m1;
    return Acc{m.m1 * b.P1, m.m0 * b.P0, s * b.Ps, fmaf(m.m0, b.Ps, m.m1 * b.D), fmaf(m.m1, b.Ps, m.m0 * b.D0)};
}

__device__ __forceinline__ Acc acc_concat(const Acc &a, const Acc &b)
{
    return Acc{a.P1 * b.P1, a.P0 * b.P0, a.Ps * b.Ps, fmaf(a.D, b.Ps, a.P1 * b.D), fmaf(a.D0, b.Ps, a.P0 * b.D0)};
}

constexpr int kAccFloats = 5;
constexpr int kLinearMaxFan = 64;  // wider factors use the per-target loop

// Phase 2 for one factor, O(n): outputs replace the old values in io.
__device__ __forceinline__ void factor_linear(int type, float p, int n, const float *in, float *io, float *pre,
                                              int stride, float &rmax, unsigned long long &ng)
{
    const unsigned t = 1u << type;
    constexpr unsigned AND = 1u << kTypeAND, OR = 1u << kTypeOR, NOT = 1u << kTypeNOT, EQ = 1u << kTypeEQ,
                       NI = 1u << kTypeNOISY_IMPLY, NA = 1u << kTypeNOISY_AND, PR = 1u << kTypePRIOR;
    const float q = 1.f - p;
    const int y = n - 1;
    Acc acc = acc_one();
    for (int j = 0; j < y; ++j) {
        pre[j] = acc.P1;
        pre[stride + j] = acc.P0;
        pre[2 * stride + j] = acc.Ps;
        pre[3 * stride + j] = acc.D;
        pre[4 * stride + j] = acc.D0;
        acc = acc_append(acc, dec(in[j]));
    }
    {   // the output (or only) variable
        const float a0 = (t & NOT) ? 1.f : (t & (NA | NI | PR)) ? q : 0.f;
        const float a1 = (t & (AND | NA | NI)) ? 1.f : 0.f;
        const float a2 = (t & (OR | EQ)) ? 1.f : 0.f;
        const float b0 = (t & (AND | EQ)) ? 1.f : (t & (NA | NI | PR)) ? p : 0.f;
        const float b1 = (t & NI) ? 1.f : 0.f;
        const float b2 = (t & OR) ? 1.f : 0.f;
        const float b3 = (t & NOT) ? 1.f : 0.f;
        const P2 mu{fmaf(a0, acc.P1, fmaf(a1, acc.D, a2 * acc.P0)),
                    fmaf(b0, acc.P1, fmaf(b1, acc.D, fmaf(b2, acc.D0, b3 * acc.P0)))};
        bool gd = false;
        const float r = enc_fast(mu, gd);
        ng += gd;
        rmax = fmaxf(rmax, delta_p1_fast(r, io[y]));
        io[y] = r;
    }
    if (y == 0) return;
    const P2 my = dec(in[y]);
    const float sy = my.m0 + my.m1, w = fmaf(p, my.m1, q * my.m0);
    const float c0 = (t & (AND | NA)) ? my.m0 : (t & NOT) ? my.m1 : (t & NI) ? sy : 0.f;
    const float c1 = (t & (OR | EQ)) ? my.m0 : 0.f;
    const float c2 = (t & OR) ? my.m1 : 0.f;
    const float d0 = (t & (AND | EQ)) ? my.m1 : (t & (NA | NI)) ? w : 0.f;
    const float d1 = (t & (AND | NA)) ? my.m0 : (t & NI) ? sy : 0.f;
    const float d2 = (t & OR) ? my.m1 : (t & NOT) ? my.m0 : 0.f;
    Acc suf = acc_one();
    for (int j = y - 1; j >= 0; --j) {
        const Acc pr{pre[j], pre[stride + j], pre[2 * stride + j], pre[3 * stride + j], pre[4 * stride + j]};
        const Acc ex = acc_concat(pr, suf);
        const P2 mu{fmaf(c0, ex.Ps, fmaf(c1, ex.P0, c2 * ex.D0)), fmaf(d0, ex.P1, fmaf(d1, ex.D, d2 * ex.Ps))};
        bool gd = false;
        const float r = enc_fast(mu, gd);
        ng += gd;
        const float mj = in[j];
        rmax = fmaxf(rmax, delta_p1_fast(r, io[j]));
        io[j] = r;
        suf = acc_prepend(dec(mj), suf);
    }
}

__global__ void __launch_bounds__(256) k_a2v_rows(const DevGraph g, const FloodPlanDev F,
                                                  const float *__restrict__ v2a, float *__restrict__ a2v,
                                                  IterCtl ctl, int staged)
{
    if (*(volatile const int *)F.done) return;
    extern __shared__ float s_dyn[];
    const int a0 = blockIdx.x * blockDim.x, a1 = min(a0 + (int)blockDim.x, g.na);
    const int e0 = __ldg(g.fptr + a0), e1 = __ldg(g.fptr + a1);
    const int cnt = e1 - e0;
    float *s_in = s_dyn, *s_io = s_dyn + staged, *s_pre = s_dyn + 2 * staged;
    const bool st = cnt <= staged;  // block-uniform
    if (st) {
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            s_in[i] = __ldg(v2a + e0 + i);
            s_io[i] = a2v[e0 + i];
        }
        __syncthreads();
    }
    float rmax = 0.f;
    unsigned long long ng = 0;
    const int a = a0 + threadIdx.x;
    const int graph = (F.batch.n_graphs > 0 && a < a1) ? __ldg(F.fgraph + a) : -1;
    const bool frozen = graph >= 0 && __ldcg(F.batch.done + graph) != 0;
    if (a < a1 && !frozen) {
        const int lo = __ldg(g.fptr + a), n = __ldg(g.fptr + a + 1) - lo;
        const int type = __ldg(g.ftype + a);
        const float p = __ldg(g.fparam + a);
        if (st && n <= kLinearMaxFan) {
            factor_linear(type, p, n, s_in + (lo - e0), s_io + (lo - e0), s_pre + (lo - e0), staged, rmax, ng);
        } else {
            // unstaged block or very wide factor: per-target closed forms
            const float *in = st ? s_in + (lo - e0) : v2a + lo;
            float *io = st ? s_io + (lo - e0) : a2v + lo;
            for (int i = 0; i < n; ++i) {
                bool gd = false;
                const float r = enc_fast(a2v_unified(type, p, n, i, [&](int j) { return dec(in[j]); }), gd);
                ng += gd;
                rmax = fmaxf(rmax, delta_p1_fast(r, io[i]));
                io[i] = r;
            }
        }
    }
    if (st) {
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) a2v[e0 + i] = s_io[i];
    }
    if (ng) atomicAdd(ctl.guards, ng);
    if (F.batch.n_graphs > 0) {
        // per-graph residual: one atomic per graph present in the warp
        const unsigned grp = __match_any_sync(0xffffffffu, graph);
        const unsigned bits = __reduce_max_sync(grp, __float_as_uint(rmax));
        if (graph >= 0 && (threadIdx.x & 31) == __ffs(grp) - 1 && bits) atomicMax(F.batch.res + graph, bits);
        return;
    }
    const float bm = block_max(rmax);
    if (threadIdx.x == 0 && bm > 0.f) atomicMax(ctl.res + (blockIdx.x % kResSlots), __float_as_uint(bm));
}

// End of an iteration of a batch: per-graph bookkeeping as in the persistent
// engine; the run is done when no graph is running.
__global__ void k_flood_batch_check(BatchCtl B, int it, int *ctl)
{
    if (*(volatile int *)ctl) return;
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
        if (s_active == 0) ctl[0] = 1;
    }
}

// End of an iteration: the residual of iteration `it` is the max over the
// slots; the slots are cleared for the next iteration; the run is marked done
// at the first iteration below tol.  Later iterations of the same batch see
// the flag and return at once.
__global__ void k_flood_check(unsigned *slots, unsigned *hist, int it, float tol, int *ctl)
{
    if (*(volatile int *)ctl) return;
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
    }
}

}  // namespace

void flood_iteration(const DevGraph &g, const FloodPlanDev &F, float *a2v, float *v2a, IterCtl ctl,
                     int staged, int it, float tol, unsigned *hist, int *done, cudaStream_t s)
{
    FloodPlanDev P = F;
    P.done = done;
    if (g.nv > 0) k_v2a_lean<<<(g.nv + 255) / 256, 256, 0, s>>>(g, P, a2v, v2a);
    if (P.n_hub > 0) k_hub_partials<<<P.n_hub, 256, 0, s>>>(g, P, a2v);
    const int nb = P.nb_small + P.nb_medium + P.n_hub;
    if (nb > 0) k_v2a_rest<<<nb, 256, 0, s>>>(g, P, a2v, v2a);
    if (g.na > 0) {
        const int blocks = (g.na + 255) / 256;
        k_a2v_rows<<<blocks, 256, flood_smem_bytes(staged), s>>>(g, P, v2a, a2v, ctl, staged);
    }
    if (P.batch.n_graphs > 0) k_flood_batch_check<<<1, 1024, 0, s>>>(P.batch, it, done);
    else k_flood_check<<<1, kResSlots, 0, s>>>(ctl.res, hist, it, tol, done);
}

size_t flood_smem_bytes(int staged) { return (size_t)staged * (2 + kAccFloats) * sizeof(float); }

// The dynamic shared-memory limit is a property of the kernel, shared by every
// graph: it only ever grows, so a graph never lowers it under another's launch.
void flood_prepare(size_t smem_bytes)
{
    static size_t current = 0;
    if (smem_bytes > current) {
        cudaFuncSetAttribute(k_a2v_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
        current = smem_bytes;
    }
}

}  // namespace fbp
