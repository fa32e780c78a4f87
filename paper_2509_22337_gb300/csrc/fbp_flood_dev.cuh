// Device-side pieces of the flooding iteration (fbp_flood.cu), shared by the
// flooding kernels and by the batch-queue kernel, which runs whole flooding
// members inside one persistent launch.  Every piece works on one item (a
// sub-chunk, a variable, a row, a warp of factors, an edge) given by index,
// so a kernel can map items to threads by block index or by a strided loop.
// kC selects coherent loads (ld.global.cg) for the data a persistent kernel
// rewrites between its phases (the variable-major messages, the beliefs, the
// sub-chunk products, the messages): the separate kernels of a flooding
// iteration read them through the non-coherent cache, which is only valid
// across kernel launches.
#pragma once

#include "fbp_msg.cuh"
#include "fbp_flood.h"

namespace fbp {
namespace fdev {
namespace {  // internal linkage: every translation unit that includes this has its own copy

__device__ __forceinline__ XP xp_one() { return XP{1.f, 1.f, 0, 0, 0, 0}; }

// In a batch, rows and factors of graphs that have stopped are skipped.
__device__ __forceinline__ bool var_frozen(const FloodPlanDev &F, int v)
{
    return F.batch.n_graphs > 0 && __ldcg(F.batch.done + __ldg(F.vgraph + v)) != 0;
}

// x in (0, 1] as mantissa * 2^exponent with the mantissa in [1, 2): integer
// operations for a normal x, frexpf (out of line) for a subnormal one.
__device__ __noinline__ float2 split_subnormal(float x)
{
    int ex;
    const float m = frexpf(x, &ex);  // [1/2, 1)
    return make_float2(2.f * m, __int_as_float(ex - 1));
}

__device__ __forceinline__ float split(float x, int &ex)
{
    const int bits = __float_as_int(x);
    ex = (bits >> 23) - 127;
    if (ex == -127) {
        const float2 me = split_subnormal(x);
        ex = __float_as_int(me.y);
        return me.x;
    }
    return __int_as_float((bits & 0x007fffff) | 0x3f800000);
}

// Multiply entry (m, e, z), mantissa m in [1, 2), by x in [0, 1]: exact zeros
// are counted; the product of the mantissas rounds the exact product once and
// is halved (exactly) back into [1, 2), so nothing ever goes subnormal.
__device__ __forceinline__ void xmul1(float &m, int &e, int &z, float x)
{
    if (x == 0.f) {
        ++z;
        return;
    }
    int ex;
    const float mx = split(x, ex);
    m *= mx;
    e += ex;
    if (m >= 2.f) {
        m *= 0.5f;
        e += 1;
    }
}

// Multiply by a rho-encoded message: its larger entry is 1, so only the
// other entry multiplies.
__device__ __forceinline__ void xmul(XP &t, float rho)
{
    const bool neg = signbit(rho);  // (1, |rho|), else (|rho|, 1)
    float m = neg ? t.m1 : t.m0;
    int e = neg ? t.e1 : t.e0, z = neg ? t.z1 : t.z0;
    xmul1(m, e, z, fabsf(rho));
    if (neg) {
        t.m1 = m; t.e1 = e; t.z1 = z;
    } else {
        t.m0 = m; t.e0 = e; t.z0 = z;
    }
}

// Product of two partial products (mantissas in [1, 2): the product rounds
// once and is halved back into [1, 2) exactly).
__device__ __forceinline__ XP xcombine(const XP &a, const XP &b)
{
    XP r;
    r.m0 = a.m0 * b.m0;
    r.m1 = a.m1 * b.m1;
    r.e0 = a.e0 + b.e0;
    r.e1 = a.e1 + b.e1;
    if (r.m0 >= 2.f) {
        r.m0 *= 0.5f;
        r.e0 += 1;
    }
    if (r.m1 >= 2.f) {
        r.m1 *= 0.5f;
        r.e1 += 1;
    }
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

// Butterfly product over the warp; multiplication commutes, so every lane
// ends with the same bits.
__device__ __forceinline__ XP warp_product(XP t)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = xcombine(t, xshfl_xor(t, o));
    return t;
}

// Belief record: the belief's two entries as the ratio b0/b1.
//   x = bits of q = m0/m1 of the mantissas (both lie in [1, 2), so q lies in
//       (1/2, 2)),
//   y = (e0 - e1) * 16 + min(z0, 2) * 4 + min(z1, 2): the exponent
//       difference (clamped to +-2^26; anything beyond +-400 saturates the
//       final message anyway) and the zero counts (two tell "zero even
//       without the own message" as well as any larger count).
__device__ __forceinline__ uint2 belief_pack(const XP &t)
{
    const float q = t.m0 * rcp_normal(t.m1);  // within a few ulp of the quotient
    const int de = max(-(1 << 26), min(1 << 26, t.e0 - t.e1));
    return make_uint2(__float_as_uint(q), (unsigned)(de * 16 + min(t.z0, 2) * 4 + min(t.z1, 2)));
}

// t * 2^k for t in (1/4, 4) and k <= 1.  While 2^k is normal this is one
// multiplication by it (exact unless the result is subnormal, where it rounds
// once); below that, two (k is clamped at -300, where every result is 0).
__device__ __forceinline__ float scale_down(float t, int k)
{
    k = max(k, -300);
    const int k1 = max(k, -126), k2 = max(k - k1, -126);
    return t * __int_as_float((127 + k1) << 23) * __int_as_float((127 + k2) << 23);
}

// v->a message of an edge whose variable has belief record b and whose own
// incoming a->v message is rho (Eq. 1: phi times every other incoming
// message, i.e. the belief without the own message), encoded; zero mass
// becomes the uniform message.  With the own message's entries x0, x1 the
// result's ratio is (b0/b1) / (x0/x1) = t 2^E with t in (1/4, 4); a zero own
// entry was counted in the belief rather than multiplied, so it divides out
// as 1.  Mantissas and exponents are split with integer operations; the
// quotient and the final reciprocal go through the approximate reciprocal
// (a few ulp) of a number in (1/4, 4).
__device__ __forceinline__ float v2a_from_belief(uint2 b, float rho)
{
    const int w = (int)b.y;
    const float a = fabsf(rho);
    const bool neg = signbit(rho);  // own message (1, a), else (a, 1)
    float t = __uint_as_float(b.x);  // in (1/2, 2)
    int E = w >> 4;
    if ((w & 15) != 0 || a == 0.f) {  // zeros counted, or a hard own message
        const int z0 = ((w >> 2) & 3) - (!neg && a == 0.f);
        const int z1 = (w & 3) - (neg && a == 0.f);
        if (z0 > 0 && z1 > 0) return 1.f;  // zero mass: uniform
        if (z0 > 0) return 0.f;            // hard (0, 1)
        if (z1 > 0) return -0.f;           // hard (1, 0)
        // here a == 0: the own zero entry divides out
    } else {
        int ea;
        const float ma = split(a, ea);  // [1, 2)
        t = neg ? t * ma : t * rcp_normal(ma);
        E += neg ? ea : -ea;
    }
    // the ratio t 2^E is at most 1 iff t 2^clamp(E, -2, 2) is (t lies in (1/4, 4))
    const bool le = t * __int_as_float((127 + max(-2, min(2, E))) << 23) <= 1.f;
    const float r = scale_down(le ? t : rcp_normal(t), le ? E : -E);
    return le ? r : -r;  // m1 the larger entry, else m0
}

template <bool kC>
__device__ __forceinline__ float ldm(const float *p)
{
    return kC ? __ldcg(p) : __ldg(p);
}

template <bool kC>
__device__ __forceinline__ uint2 ldb(const uint2 *p)
{
    return kC ? __ldcg(p) : __ldg(p);
}

// An XP record (24 bytes: three 8-byte-aligned pairs).
template <bool kC>
__device__ __forceinline__ XP ldx(const XP *p)
{
    if (!kC) return *p;
    const float2 m = __ldcg(reinterpret_cast<const float2 *>(&p->m0));
    const int2 e = __ldcg(reinterpret_cast<const int2 *>(&p->e0));
    const int2 z = __ldcg(reinterpret_cast<const int2 *>(&p->z0));
    return XP{m.x, m.y, e.x, e.y, z.x, z.y};
}

// Product of entries x[b, end) in order (at most one sub-chunk), one thread;
// entries load in groups of four, each group while the one before it
// multiplies (few registers: this shares a launch with latency-bound work
// that wants every warp slot).  Entries past the warp's longest run are
// skipped by a uniform branch (a padded entry would multiply by exactly 1).
template <bool kC>
__device__ __forceinline__ XP seq_product(const float *__restrict__ x, int b, int end)
{
    constexpr int kG = 4;
    const int nw = __reduce_max_sync(__activemask(), end - b);
    float r[kG], nx[kG];
#pragma unroll
    for (int u = 0; u < kG; ++u) r[u] = b + u < end ? ldm<kC>(x + b + u) : 1.f;
    XP t = xp_one();
#pragma unroll
    for (int gi = 0; gi < kFloodSub / kG; ++gi) {
        const int c = b + (gi + 1) * kG;  // first entry of the next group
#pragma unroll
        for (int u = 0; u < kG; ++u) nx[u] = 1.f;
        if (gi + 1 < kFloodSub / kG && (gi + 1) * kG < nw) {
#pragma unroll
            for (int u = 0; u < kG; ++u) nx[u] = c + u < end ? ldm<kC>(x + c + u) : 1.f;
        }
#pragma unroll
        for (int u = 0; u < kG; ++u)
            if (gi * kG + u < nw) xmul(t, r[u]);
#pragma unroll
        for (int u = 0; u < kG; ++u) r[u] = nx[u];
    }
    return t;
}

// ---------------------------------------------------------------------------
// Phase 1 items
// ---------------------------------------------------------------------------
// Sub-chunk k of the rows longer than 8 entries: its product; a row of one
// sub-chunk gets its belief here.
template <bool kC>
__device__ __forceinline__ void sub_product_item(const DevGraph &g, const FloodPlanDev &F,
                                                 const float *__restrict__ a2v_vm, int k)
{
    const int4 sc = __ldg(F.subs + k);  // {variable, begin, end, agg slot or -1}
    if (var_frozen(F, sc.x)) return;
    XP t = seq_product<kC>(a2v_vm, sc.y, sc.z);
    if (sc.w >= 0) {
        F.agg[sc.w] = t;
        return;
    }
    xmul(t, __ldg(g.phi + sc.x));
    F.belief[sc.x] = belief_pack(t);
}

// Variable v of degree <= 8 (others return): its belief, entries in row
// order.  Slots past the longest row among the calling warp's active lanes
// are skipped by a uniform branch (a padded slot would multiply by exactly 1).
template <bool kC>
__device__ __forceinline__ void belief_short_row(const FloodPlanDev &F, const float *__restrict__ a2v_vm, int v, int lo,
                                                 int d, float phi)
{
    const int dw = __reduce_max_sync(__activemask(), d);
    float r[kFloodSmallMax];
#pragma unroll
    for (int u = 0; u < kFloodSmallMax / 2; ++u) r[u] = u < d ? ldm<kC>(a2v_vm + lo + u) : 1.f;
    if (dw > kFloodSmallMax / 2) {
#pragma unroll
        for (int u = kFloodSmallMax / 2; u < kFloodSmallMax; ++u) r[u] = u < d ? ldm<kC>(a2v_vm + lo + u) : 1.f;
    }
    XP t = xp_one();
#pragma unroll
    for (int u = 0; u < kFloodSmallMax; ++u)
        if (u < dw) xmul(t, r[u]);
    xmul(t, phi);
    F.belief[v] = belief_pack(t);
}

template <bool kC>
__device__ __forceinline__ void belief_var_item(const DevGraph &g, const FloodPlanDev &F,
                                                const float *__restrict__ a2v_vm, int v)
{
    if (var_frozen(F, v)) return;
    const int lo = __ldg(g.vptr + v), d = __ldg(g.vptr + v + 1) - lo;
    if (d > kFloodSmallMax) return;  // a row of sub-chunks
    belief_short_row<kC>(F, a2v_vm, v, lo, d, __ldg(g.phi + v));
}

// The same for variables v, v + stride, ... below g.nv, one thread: the next
// variable's row bounds and phi load while this one's row multiplies.
__device__ __forceinline__ void belief_var_loop(const DevGraph &g, const FloodPlanDev &F,
                                                const float *__restrict__ a2v_vm, int v, int stride)
{
    int lo = 0, d = 0;
    float phi = 1.f;
    if (v < g.nv) {
        lo = __ldg(g.vptr + v);
        d = __ldg(g.vptr + v + 1) - lo;
        phi = __ldg(g.phi + v);
    }
    while (v < g.nv) {
        const int vn = v + stride;
        int lo_n = 0, d_n = 0;
        float phi_n = 1.f;
        if (vn < g.nv) {
            lo_n = __ldg(g.vptr + vn);
            d_n = __ldg(g.vptr + vn + 1) - lo_n;
            phi_n = __ldg(g.phi + vn);
        }
        if (d <= kFloodSmallMax && !var_frozen(F, v)) belief_short_row<false>(F, a2v_vm, v, lo, d, phi);
        v = vn;
        lo = lo_n;
        d = d_n;
        phi = phi_n;
    }
}

// Medium row w (2..8 sub-chunks): the butterfly over the slots of which slots
// 0..ns-1 hold sub-chunk products (the others the identity), evaluated by one
// thread: slot 0 ends with ((P0 P4)(P2 P6)) ((P1 P5)(P3 P7)); a product with
// the identity is the value itself, so missing sub-chunks are skipped.
template <bool kC>
__device__ __forceinline__ void belief_medium_row(const DevGraph &g, const FloodPlanDev &F, const int4 row)
{
    // row = {variable, first agg slot, sub-chunks (2..8), 0}
    if (var_frozen(F, row.x)) return;
    const XP *P = F.agg + row.y;
    const int ns = row.z;
    XP t = ldx<kC>(P);
    if (ns > 4) t = xcombine(t, ldx<kC>(P + 4));
    if (ns > 2) {
        XP u = ldx<kC>(P + 2);
        if (ns > 6) u = xcombine(u, ldx<kC>(P + 6));
        t = xcombine(t, u);
    }
    XP u = ldx<kC>(P + 1);
    if (ns > 5) u = xcombine(u, ldx<kC>(P + 5));
    if (ns > 3) {
        XP u3 = ldx<kC>(P + 3);
        if (ns > 7) u3 = xcombine(u3, ldx<kC>(P + 7));
        u = xcombine(u, u3);
    }
    t = xcombine(t, u);
    xmul(t, __ldg(g.phi + row.x));
    F.belief[row.x] = belief_pack(t);
}

template <bool kC>
__device__ __forceinline__ void belief_medium_item(const DevGraph &g, const FloodPlanDev &F, int w)
{
    belief_medium_row<kC>(g, F, __ldg(F.medium + w));
}

// Hub row hr, one whole block of kFloodSlots threads: thread j combines
// sub-chunks j, j + kFloodSlots, ... in order, keeping the next kD of them in
// flight (the chain, not the arithmetic, sets the time; kD only trades
// registers for that), then the xor butterfly over the slots: j with j^128,
// j^64, j^32 through shared memory s_x (kFloodSlots records), the rest by
// shuffle in warp 0.  Every thread of the block calls it with the same hr.
template <bool kC, int kD>
__device__ __forceinline__ void belief_hub_block(const DevGraph &g, const FloodPlanDev &F, int hr, XP *s_x)
{
    const int j0 = threadIdx.x;
    const int4 row = __ldg(F.hub_row + hr);  // {variable, first agg slot, sub-chunks, 0}
    if (var_frozen(F, row.x)) return;        // block-uniform
    const XP *P = F.agg + row.y;
    const int n = row.z;
    XP buf[kD];
#pragma unroll
    for (int d = 0; d < kD; ++d) buf[d] = j0 + kFloodSlots * d < n ? ldx<kC>(P + j0 + kFloodSlots * d) : xp_one();
    XP t = xp_one();
    for (int base = 0; base < n; base += kFloodSlots * kD) {  // block-uniform
#pragma unroll
        for (int d = 0; d < kD; ++d) {
            const int j = base + kFloodSlots * d + j0, jn = j + kFloodSlots * kD;
            if (j < n) t = xcombine(t, buf[d]);
            if (jn < n) buf[d] = ldx<kC>(P + jn);
        }
    }
#pragma unroll
    for (int k = kFloodSlots / 2; k >= 32; k >>= 1) {
        s_x[j0] = t;
        __syncthreads();
        if (j0 < k) t = xcombine(t, s_x[j0 + k]);
        __syncthreads();
    }
    if (j0 < 32) {
        t = warp_product(t);
        if (j0 == 0) {
            xmul(t, __ldg(g.phi + row.x));
            F.belief[row.x] = belief_pack(t);
        }
    }
}

// ---------------------------------------------------------------------------
// Phase 2 items
// ---------------------------------------------------------------------------
// Per-graph residual of a batch: one atomic per graph present in the warp.
__device__ __forceinline__ void batch_residual(const FloodPlanDev &F, int graph, float d)
{
    const unsigned grp = __match_any_sync(0xffffffffu, graph);
    const unsigned bits = __reduce_max_sync(grp, __float_as_uint(d));
    if (graph >= 0 && (threadIdx.x & 31) == __ffs(grp) - 1 && bits) max_bits(F.batch.res + graph, bits);
}

// Typed factors of at most 32 variables: one lane per message, each warp
// holding whole consecutive factors (so its edges are one contiguous range and
// every streamed load and store is coalesced).  The warp reads its factors'
// row offsets, types and parameters once (lane j: factor j) and each lane
// finds its factor from the mask of factor starts.  A lane forms its own v->a
// message from its variable's belief and its edge's current a->v message; the
// closed forms (Eq. 4 with the common products factored out) then need three
// products over the factor's premises other than the lane's own:
//   X = prod m_j1,  Y = prod s_j (s_j = m_j0 + m_j1),
//   D = sum_k (prod_{j<k} m_j1) m_k0 (prod_{j>k} s_j)  (= Y - X, no cancellation),
// accumulated in premise order from the neighbouring lanes' messages by
// shuffle, over a trip count that is uniform in the warp.  With the output's
// incoming message my and p the factor's parameter (q = 1-p):
//   type         to the output             to a premise
//   AND          (D, X)                    (my0 Y, my1 X + my0 D)
//   NOISY_AND    (qX + D, pX)              (my0 Y, (p my1 + q my0) X + my0 D)
//   NOISY_IMPLY  (qX + D, pX + D)          (sy Y, (p my1 + q my0) X + sy D), sy = my0 + my1
//   PRIOR        NOISY_AND with no premise: (q, p)
//   OR           AND with every incoming message and the result flipped
//                (x -> 1-x is a bijection that maps OR onto AND)
//   NOT          AND with one premise and the result flipped
//   EQ           every variable is a "premise", s_j replaced by m_j0:
//                to variable i (Y, X) = (prod_{u != i} m_u0, prod_{u != i} m_u1)
// Messages enter scaled so that their larger entry is 1, so Y <= 2^31.
// Each lane decodes its own v->a message once (flipped for OR) and the
// others' arrive decoded by shuffle.
// Called by a whole warp with the same w; returns the lane's |dP(x=1)| in dd
// (0 for no write), its guard count in ng and (batch) its graph.  kFeat
// selects the optional parts: kFeatBatch (a batched union: factors of
// finished graphs are skipped, graph returned), kFeatLevel (one level of a
// device-scheduled RESIDUAL iteration: only edges with F.elevel[e] ==
// F.level are written), kFeatDres (each written edge's |dP| is recorded in
// F.dres).
constexpr int kFeatBatch = 1, kFeatLevel = 2, kFeatDres = 4;
template <bool kC, int kFeat>
__device__ __forceinline__ void lanes_warp(const DevGraph &g, const FloodPlanDev &F, float *__restrict__ a2v,
                                           float *__restrict__ a2v_vm, int w, float &dd, unsigned long long &ng,
                                           int &graph)
{
    const int lane = threadIdx.x & 31;
    const int4 wr = __ldg(F.twarps + w);  // {first edge, end edge, first factor, end factor}
    const int nf = wr.w - wr.z, ne_w = wr.y - wr.x;
    int fst = 0, ftyp = 0, fgr = -1;
    float fpar = 0.f;
    if (lane < nf) {
        fst = __ldg(g.fptr + wr.z + lane) - wr.x;
        ftyp = __ldg(g.ftype + wr.z + lane);
        fpar = __ldg(g.fparam + wr.z + lane);
        if constexpr ((kFeat & kFeatBatch) != 0) fgr = __ldg(F.fgraph + wr.z + lane);
    }
    const unsigned starts = __reduce_or_sync(0xffffffffu, lane < nf ? 1u << fst : 0u);
    const unsigned upto = starts & (0xffffffffu >> (31 - lane));  // factor starts at or before this lane
    const int fi = __popc(upto) - 1;                              // this lane's factor in the warp
    const int first = 31 - __clz(upto);                           // lane of its first edge
    const unsigned after = starts & ~(0xffffffffu >> (31 - lane));
    const bool valid = lane < ne_w;
    const int n = (after ? __ffs(after) - 1 : ne_w) - first;
    const int type = __shfl_sync(0xffffffffu, ftyp, fi);
    const float p = __shfl_sync(0xffffffffu, fpar, fi), q = 1.f - p;
    const bool eq = type == kTypeEQ, fin = type == kTypeOR, fout = type == kTypeOR || type == kTypeNOT;
    const int i = lane - first, np = eq ? n : n - 1;
    const int e = wr.x + lane;
    float x = 1.f, old = 1.f;
    int slot = 0;
    bool frozen = false;
    if constexpr ((kFeat & kFeatBatch) != 0) {
        graph = __shfl_sync(0xffffffffu, fgr, fi);
        frozen = __ldcg(F.batch.done + graph) != 0;
    }
    if (valid) {
        const int v = __ldcs(g.fvars + e);
        slot = __ldcs(F.vpos + e);
        old = kC ? __ldcg(a2v + e) : __ldcs(a2v + e);
        x = v2a_from_belief(ldb<kC>(F.belief + v), old);
    } else {
        graph = -1;
    }
    // this lane's message decoded (flipped with the inputs for OR), and the
    // entry that multiplies Y
    P2 me = dec(x);
    if (fin) me = P2{me.m1, me.m0};
    const float ey_me = eq ? me.m0 : me.m0 + me.m1;
    // the output's message
    const int last = (first + n - 1) & 31;
    P2 my{__shfl_sync(0xffffffffu, me.m0, last), __shfl_sync(0xffffffffu, me.m1, last)};
    if (eq) my = P2{1.f, 1.f};
    float X = 1.f, Y = 1.f, D = 0.f;
    const int span = __reduce_max_sync(0xffffffffu, valid ? np : 0);
#pragma unroll 2
    for (int j = 0; j < span; ++j) {
        const int src = (first + j) & 31;
        const float m0 = __shfl_sync(0xffffffffu, me.m0, src), m1 = __shfl_sync(0xffffffffu, me.m1, src);
        const float ey = __shfl_sync(0xffffffffu, ey_me, src);
        if (j < np && j != i) {
            D = fmaf(D, ey, X * m0);
            X *= m1;
            Y *= ey;
        }
    }
    const bool nz = type == kTypeNOISY_AND || type == kTypePRIOR, ni = type == kTypeNOISY_IMPLY;
    P2 mu;
    if (i == np) {  // the output: mu0 = a0 X + D, mu1 = b0 X + b1 D
        const float a0 = (nz || ni) ? q : 0.f, b0 = (nz || ni) ? p : 1.f, b1 = ni ? 1.f : 0.f;
        mu = P2{fmaf(a0, X, D), fmaf(b0, X, b1 * D)};
    } else {        // a premise: mu0 = c0 Y, mu1 = d0 X + d1 D
        const float sy = my.m0 + my.m1, wq = fmaf(p, my.m1, q * my.m0);
        const float c0 = eq ? 1.f : ni ? sy : my.m0;
        const float d0 = eq ? 1.f : (nz || ni) ? wq : my.m1;
        const float d1 = eq ? 0.f : ni ? sy : my.m0;
        mu = P2{c0 * Y, fmaf(d0, X, d1 * D)};
    }
    if (fout) mu = P2{mu.m1, mu.m0};
    bool write = valid && !frozen;
    if constexpr ((kFeat & kFeatLevel) != 0) write = write && __ldg(F.elevel + e) == F.level;
    if (write) {
        bool gd = false;
        const float r = enc_fast(mu, gd);
        ng += gd;
        dd = delta_p1_fast(r, old);
        a2v[e] = r;  // a plain store: the next iteration's phase 2 reads it back, and L2 may keep it
        a2v_vm[slot] = r;
        if constexpr ((kFeat & kFeatDres) != 0) F.dres[e] = dd;
    }
}

// v->a message of wide-list entry k (an edge of a factor wider than a warp),
// formed before the factor's a->v messages are (those are written in place).
template <bool kC>
__device__ __forceinline__ void wide_v2a_item(const DevGraph &g, const FloodPlanDev &F, const float *__restrict__ a2v,
                                              int k)
{
    const int e = __ldg(F.wide + k);
    F.wide_v2a[k] = v2a_from_belief(ldb<kC>(F.belief + __ldg(g.fvars + e)), ldm<kC>(a2v + e));
}

// a->v message of wide-list entry k: the closed form over the factor's v->a
// messages (consecutive in wide_v2a, factor by factor).
template <bool kC>
__device__ __forceinline__ void wide_a2v_item(const DevGraph &g, const FloodPlanDev &F, float *__restrict__ a2v,
                                              float *__restrict__ a2v_vm, int k, float &dd, unsigned long long &ng,
                                              int &graph)
{
    const int e = __ldg(F.wide + k);
    const int a = __ldg(g.efac + e);
    const int lo = __ldg(g.fptr + a), n = __ldg(g.fptr + a + 1) - lo;
    const float *xv = F.wide_v2a + (k - (e - lo));  // the factor's first edge in the wide list
    bool frozen = false;
    if (F.batch.n_graphs > 0) {
        graph = __ldg(F.fgraph + a);
        frozen = __ldcg(F.batch.done + graph) != 0;
    }
    if (frozen || (F.elevel && __ldg(F.elevel + e) != F.level)) return;
    const int type = __ldg(g.ftype + a);
    const P2 mu = type == kTypeTERMS
                      ? a2v_terms(g, a, n, e - lo, [&](int j) { return dec(ldm<kC>(xv + j)); })
                      : a2v_unified(type, __ldg(g.fparam + a), n, e - lo, [&](int j) { return dec(ldm<kC>(xv + j)); });
    bool gd = false;
    const float r = enc_fast(mu, gd);
    ng += gd;
    const float old = ldm<kC>(a2v + e);
    dd = delta_p1_fast(r, old);
    a2v[e] = r;
    a2v_vm[__ldg(F.vpos + e)] = r;
    if (F.dres) F.dres[e] = dd;
}

}  // namespace
}  // namespace fdev
}  // namespace fbp
