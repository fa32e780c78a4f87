// Flooding (PARALL) iteration kernels (sm_103a), for graphs of any degree
// distribution (BINGO-shaped derivation graphs have hub variables with 1e5
// incident factors next to millions of degree-2 variables).
//
// Phase 1, Eq. (1) in belief form: every variable's belief
//   b_v = phi_v * prod_{a in N(v)} mu_{a->v}
// is reduced once, from a variable-major copy of the a->v messages that each
// row reads contiguously, and stored as a compact ratio record (8 bytes);
// mu_{v->a} = b_v / mu_{a->v} is then formed where phase 2 needs it.  This is
// exact in the algebra of the messages as long as (i) exact zeros (hard
// messages) are counted rather than multiplied in, and (ii) the product never
// underflows: each of the two entries is kept as a mantissa and an integer
// exponent while the row is reduced.
//   rows of degree <= 8       one thread per row, entries in row order
//   longer rows               one thread per 32-entry sub-chunk; a row of
//                             2..8 sub-chunks (at most FBP_OPT_FLOOD_HUB_MIN
//                             entries) combined by one thread, a longer one
//                             by one warp
// The product of every row longer than 8 entries is grouped one way only,
// whichever kernel carries the row: the row is cut into 32-entry sub-chunks,
// each multiplied in order; sub-chunk s goes to slot s mod 32 (a slot
// multiplies its sub-chunks in order), and the 32 slots are combined by an
// xor butterfly (slot j with slot j^16, then j^8, j^4, j^2, j^1).  A row of at
// most 256 entries fills slots 0..7 only, and the one-thread combine
// evaluates exactly that butterfly, so the thread and the warp combines
// compute the same bits and the split options (FBP_OPT_FLOOD_HUB_MIN,
// _CHUNK) only move work between kernels.  phi_v is multiplied in last.  Every multiply
// rounds the exact product once (the mantissa/exponent form never goes
// subnormal), so only this grouping decides the result.
//
// Phase 2, the closed-form local-structure messages (Eq. 4).  Every v->a
// message is formed from its variable's belief and the edge's current a->v
// message; the new a->v message is written in place (factor-major) and into
// the variable-major copy.  Factors of at most 32 variables: one lane per
// message, whole consecutive factors per warp, the factor's other messages by
// warp shuffle (typed factors in one kernel, generic ones in another).
// Factors wider than a warp: one thread per edge.
//
// Memory traffic per iteration: phase 1 streams the variable-major copy,
// the row offsets and phi and writes one record per variable; phase 2
// streams the factor-major variables, the variable-major slots and the
// messages (read and write), gathers one belief record per edge (an array of
// 8 bytes per variable, small enough to stay in L2) and scatters one message
// per edge into the variable-major copy.
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
    const float q = t.m0 * rcp_approx(t.m1);  // within a few ulp of the quotient
    const int de = max(-(1 << 26), min(1 << 26, t.e0 - t.e1));
    return make_uint2(__float_as_uint(q), (unsigned)(de * 16 + min(t.z0, 2) * 4 + min(t.z1, 2)));
}

// r * 2^E by two exact power-of-two factors (each exponent clamped to the
// normal range), so a result in the normal range rounds once; far outside it
// the result saturates to 0 or infinity, as the exact one would in FP32.
__device__ __forceinline__ float scale2(float r, int E)
{
    E = max(-300, min(300, E));
    const int e1 = E / 2, e2 = E - e1;
    r *= __int_as_float((127 + max(-126, min(127, e1))) << 23);
    return r * __int_as_float((127 + max(-126, min(127, e2))) << 23);
}

// v->a message of an edge whose variable has belief record b and whose own
// incoming a->v message is rho (Eq. 1: phi times every other incoming
// message, i.e. the belief without the own message), encoded; zero mass
// becomes the uniform message.  With the own message's entries x0, x1 the
// result's ratio is (b0/b1) / (x0/x1); a zero own entry was counted in the
// belief rather than multiplied, so it divides out as 1.  Mantissas and
// exponents are split with integer operations; quotients go through the
// approximate reciprocal (a few ulp).
__device__ __forceinline__ float v2a_from_belief(uint2 b, float rho)
{
    const int w = (int)b.y;
    const float a = fabsf(rho);
    const bool neg = signbit(rho);  // own message (1, a), else (a, 1)
    const int z0 = ((w >> 2) & 3) - (!neg && a == 0.f);
    const int z1 = (w & 3) - (neg && a == 0.f);
    if (z0 > 0 && z1 > 0) return 1.f;  // zero mass: uniform
    if (z0 > 0) return 0.f;            // hard (0, 1)
    if (z1 > 0) return -0.f;           // hard (1, 0)
    float r = __uint_as_float(b.x);    // in (1/2, 2)
    int E = w >> 4;
    if (a != 0.f) {
        int ea;
        const float ma = split(a, ea);  // [1, 2)
        r = neg ? r * ma : r * rcp_approx(ma);
        E += neg ? ea : -ea;
    }
    r = scale2(r, E);
    if (r <= 1.f) return r;            // m1 is the larger entry
    return -rcp_approx(r);             // m0 is the larger entry
}

// Product of entries x[b, end) in order (at most one sub-chunk), one thread;
// every load is issued first.  Entries past the warp's longest run are
// skipped by a uniform branch (a padded entry would multiply by exactly 1).
__device__ __forceinline__ XP seq_product(const float *__restrict__ x, int b, int end)
{
    float r[kFloodSub];
#pragma unroll
    for (int u = 0; u < kFloodSub; ++u) r[u] = b + u < end ? __ldg(x + b + u) : 1.f;
    const int nw = __reduce_max_sync(__activemask(), end - b);
    XP t = xp_one();
#pragma unroll
    for (int u = 0; u < kFloodSub; ++u)
        if (u < nw) xmul(t, r[u]);
    return t;
}

// ----------------------------------------------------------------------------
// Phase 1
// ----------------------------------------------------------------------------
__global__ void k_sync_vm(const DevGraph g, const float *__restrict__ a2v, float *__restrict__ a2v_vm)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < g.ne) a2v_vm[k] = a2v[__ldg(g.vedge + k)];
}

// Products of the 32-entry sub-chunks of the rows longer than 8 entries, one
// thread per sub-chunk; a row of one sub-chunk gets its belief here.
__global__ void __launch_bounds__(256) k_sub_products(const DevGraph g, FloodPlanDev F,
                                                      const float *__restrict__ a2v_vm)
{
    if (*(volatile const int *)F.done) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= F.n_subs) return;
    const int4 sc = __ldg(F.subs + k);  // {variable, begin, end, agg slot or -1}
    if (var_frozen(F, sc.x)) return;
    XP t = seq_product(a2v_vm, sc.y, sc.z);
    if (sc.w >= 0) {
        F.agg[sc.w] = t;
        return;
    }
    xmul(t, __ldg(g.phi + sc.x));
    F.belief[sc.x] = belief_pack(t);
}

// Beliefs.  Blocks [0, nb_vars): one thread per variable of degree <= 8;
// then one thread per medium row; then one warp per hub row (both combine
// sub-chunk products of k_sub_products).
__global__ void __launch_bounds__(256) k_beliefs(const DevGraph g, FloodPlanDev F, const float *__restrict__ a2v_vm)
{
    if (*(volatile const int *)F.done) return;
    const int b = blockIdx.x;
    if (b < F.nb_vars) {
        const int v = b * blockDim.x + threadIdx.x;
        if (v >= g.nv || var_frozen(F, v)) return;
        const int lo = __ldg(g.vptr + v), d = __ldg(g.vptr + v + 1) - lo;
        if (d > kFloodSmallMax) return;  // a row of sub-chunks
        const float phi = __ldg(g.phi + v);
        // slots past the warp's longest row are skipped by a uniform branch
        // (a padded slot would multiply by exactly 1)
        const int dw = __reduce_max_sync(__activemask(), d);
        float r[kFloodSmallMax];
#pragma unroll
        for (int u = 0; u < kFloodSmallMax / 2; ++u) r[u] = u < d ? __ldg(a2v_vm + lo + u) : 1.f;
        if (dw > kFloodSmallMax / 2) {
#pragma unroll
            for (int u = kFloodSmallMax / 2; u < kFloodSmallMax; ++u) r[u] = u < d ? __ldg(a2v_vm + lo + u) : 1.f;
        }
        XP t = xp_one();
#pragma unroll
        for (int u = 0; u < kFloodSmallMax; ++u)
            if (u < dw) xmul(t, r[u]);
        xmul(t, phi);
        F.belief[v] = belief_pack(t);
        return;
    }
    if (b < F.nb_vars + F.nb_medium) {
        const int w = (b - F.nb_vars) * blockDim.x + threadIdx.x;
        if (w >= F.n_medium) return;
        const int4 row = __ldg(F.medium + w);  // {variable, first agg slot, sub-chunks (2..8), 0}
        if (var_frozen(F, row.x)) return;
        const XP *P = F.agg + row.y;
        const int ns = row.z;
        // the butterfly over 32 slots of which slots 0..ns-1 hold sub-chunk
        // products (the others the identity): slot 0 ends with
        // ((P0 P4)(P2 P6)) ((P1 P5)(P3 P7)); a product with the identity is
        // the value itself, so missing sub-chunks are skipped
        XP t = P[0];
        if (ns > 4) t = xcombine(t, P[4]);
        if (ns > 2) {
            XP u = P[2];
            if (ns > 6) u = xcombine(u, P[6]);
            t = xcombine(t, u);
        }
        XP u = P[1];
        if (ns > 5) u = xcombine(u, P[5]);
        if (ns > 3) {
            XP u3 = P[3];
            if (ns > 7) u3 = xcombine(u3, P[7]);
            u = xcombine(u, u3);
        }
        t = xcombine(t, u);
        xmul(t, __ldg(g.phi + row.x));
        F.belief[row.x] = belief_pack(t);
        return;
    }
    const int hr = (b - F.nb_vars - F.nb_medium) * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (hr >= F.n_hub_rows) return;
    const int4 row = __ldg(F.hub_row + hr);  // {variable, first agg slot, sub-chunks, 0}
    if (var_frozen(F, row.x)) return;
    XP t = xp_one();
    for (int j = lane; j < row.z; j += 32) t = xcombine(t, F.agg[row.y + j]);
    t = warp_product(t);
    if (lane == 0) {
        xmul(t, __ldg(g.phi + row.x));
        F.belief[row.x] = belief_pack(t);
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
__global__ void __launch_bounds__(256) k_a2v_lanes(const DevGraph g, const FloodPlanDev F, float *__restrict__ a2v,
                                                   float *__restrict__ a2v_vm, IterCtl ctl)
{
    if (*(volatile const int *)F.done) return;
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    float dd = 0.f;
    unsigned long long ng = 0;
    int graph = -1;
    if (w < F.n_twarps) {  // warp-uniform
        const int4 wr = __ldg(F.twarps + w);  // {first edge, end edge, first factor, end factor}
        const int nf = wr.w - wr.z, ne_w = wr.y - wr.x;
        int fst = 0, ftyp = 0, fgr = -1;
        float fpar = 0.f;
        if (lane < nf) {
            fst = __ldg(g.fptr + wr.z + lane) - wr.x;
            ftyp = __ldg(g.ftype + wr.z + lane);
            fpar = __ldg(g.fparam + wr.z + lane);
            if (F.batch.n_graphs > 0) fgr = __ldg(F.fgraph + wr.z + lane);
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
        if (F.batch.n_graphs > 0) {
            graph = __shfl_sync(0xffffffffu, fgr, fi);
            frozen = __ldcg(F.batch.done + graph) != 0;
        }
        if (valid) {
            const int v = __ldcs(g.fvars + e);
            slot = __ldcs(F.vpos + e);
            old = __ldcs(a2v + e);
            x = v2a_from_belief(__ldg(F.belief + v), old);
        } else {
            graph = -1;
        }
        // the output's message (flipped with the inputs for OR)
        P2 my = dec(__shfl_sync(0xffffffffu, x, (first + n - 1) & 31));
        if (fin) my = P2{my.m1, my.m0};
        if (eq) my = P2{1.f, 1.f};
        float X = 1.f, Y = 1.f, D = 0.f;
        const int span = __reduce_max_sync(0xffffffffu, valid ? np : 0);
        for (int j = 0; j < span; ++j) {
            const float r = __shfl_sync(0xffffffffu, x, (first + j) & 31);
            if (j < np && j != i) {
                P2 m = dec(r);
                if (fin) m = P2{m.m1, m.m0};
                const float ey = eq ? m.m0 : m.m0 + m.m1;
                D = fmaf(D, ey, X * m.m0);
                X *= m.m1;
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
        if (valid && !frozen && (!F.elevel || __ldg(F.elevel + e) == F.level)) {
            bool gd = false;
            const float r = enc_fast(mu, gd);
            ng += gd;
            dd = delta_p1_fast(r, old);
            __stcs(a2v + e, r);
            a2v_vm[slot] = r;
            if (F.dres) F.dres[e] = dd;
        }
    }
    if (ng) atomicAdd(ctl.guards, ng);
    if (F.batch.n_graphs > 0) {
        batch_residual(F, graph, dd);
        return;
    }
    const float bm = block_max(dd);
    if (threadIdx.x == 0 && bm > 0.f) max_bits(ctl.res + (blockIdx.x % kResSlots), __float_as_uint(bm));
}

// Generic factors: one lane per message; each warp holds whole generic factors (consecutive in the
// factor-major order, so its edges are one contiguous range and every
// streamed load and store is coalesced).  The warp reads its factors' row
// offsets, types and parameters once (lane j: factor j) and each lane finds
// its factor from the mask of factor starts.  A lane forms its own v->a
// message from its variable's belief and its edge's current a->v message;
// the factor's other messages come from the neighbouring lanes by shuffle, in
// premise order (the order of a2v_unified, so the closed form's arithmetic is
// the level engine's), over a trip count that is uniform in the warp, so that
// factors of different types and fan-ins in one warp run one instruction
// stream.  A factor of at most 32 variables has Ps <= 2^31, so the products
// need no rescaling here.
__global__ void __launch_bounds__(256) k_a2v_fused(const DevGraph g, const FloodPlanDev F, float *__restrict__ a2v,
                                                   float *__restrict__ a2v_vm, IterCtl ctl)
{
    if (*(volatile const int *)F.done) return;
    __shared__ float s_x[256];  // the lanes' v->a messages (generic factors read them here)
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    float d = 0.f;
    unsigned long long ng = 0;
    int graph = -1;
    if (w < F.n_warps) {  // warp-uniform
        const int4 wr = __ldg(F.warps + w);  // {first edge, end edge, first factor, end factor}
        const int nf = wr.w - wr.z, ne_w = wr.y - wr.x;
        int fst = 0, ftyp = 0, fgr = -1;
        float fpar = 0.f;
        if (lane < nf) {
            fst = __ldg(g.fptr + wr.z + lane) - wr.x;
            ftyp = __ldg(g.ftype + wr.z + lane);
            fpar = __ldg(g.fparam + wr.z + lane);
            if (F.batch.n_graphs > 0) fgr = __ldg(F.fgraph + wr.z + lane);
        }
        const unsigned starts = __reduce_or_sync(0xffffffffu, lane < nf ? 1u << fst : 0u);
        const unsigned upto = starts & (0xffffffffu >> (31 - lane));  // factor starts at or before this lane
        const int fi = __popc(upto) - 1;                              // this lane's factor in the warp
        const int first = 31 - __clz(upto);                           // lane of its first edge
        const unsigned after = starts & ~(0xffffffffu >> (31 - lane));
        const bool valid = lane < ne_w;
        const int n = (after ? __ffs(after) - 1 : ne_w) - first;
        const int i = lane - first, y = n - 1;
        const int type = __shfl_sync(0xffffffffu, ftyp, fi);
        const float p = __shfl_sync(0xffffffffu, fpar, fi);
        const int e = wr.x + lane;
        float x = 1.f, old = 1.f;
        int slot = 0;
        bool frozen = false;
        if (F.batch.n_graphs > 0) {
            graph = __shfl_sync(0xffffffffu, fgr, fi);
            frozen = graph < 0 || __ldcg(F.batch.done + graph) != 0;
        }
        if (valid) {
            const int v = __ldcs(g.fvars + e);
            slot = __ldcs(F.vpos + e);
            old = __ldcs(a2v + e);
            x = v2a_from_belief(__ldg(F.belief + v), old);
        } else {
            graph = -1;
        }
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
            const int a = wr.z + fi;
            const P2 mu = type == kTypeTERMS ? a2v_terms(g, a, n, i, [&](int j) { return dec(wx[j]); })
                                             : a2v_finish(type, p, i == y, A, dec(ry));
            bool gd = false;
            const float r = enc_fast(mu, gd);
            ng += gd;
            d = delta_p1_fast(r, old);
            __stcs(a2v + e, r);
            a2v_vm[slot] = r;
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

// v->a messages of the edges of factors wider than a warp, formed before
// their a->v messages are (those are written in place).
__global__ void __launch_bounds__(256) k_wide_v2a(const DevGraph g, const FloodPlanDev F,
                                                  const float *__restrict__ a2v)
{
    if (*(volatile const int *)F.done) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= F.n_wide) return;
    const int e = __ldg(F.wide + k);
    F.wide_v2a[k] = v2a_from_belief(__ldg(F.belief + __ldg(g.fvars + e)), a2v[e]);
}

// Factors wider than a warp: one thread per edge, the closed form over the
// factor's v->a messages (consecutive in wide_v2a, factor by factor).
__global__ void __launch_bounds__(256) k_a2v_wide(const DevGraph g, const FloodPlanDev F, float *__restrict__ a2v,
                                                  float *__restrict__ a2v_vm, IterCtl ctl)
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
        const float *xv = F.wide_v2a + (k - (e - lo));  // the factor's first edge in the wide list
        bool frozen = false;
        if (F.batch.n_graphs > 0) {
            graph = __ldg(F.fgraph + a);
            frozen = __ldcg(F.batch.done + graph) != 0;
        }
        if (!frozen && (!F.elevel || __ldg(F.elevel + e) == F.level)) {
            const int type = __ldg(g.ftype + a);
            const P2 mu = type == kTypeTERMS
                              ? a2v_terms(g, a, n, e - lo, [&](int j) { return dec(xv[j]); })
                              : a2v_unified(type, __ldg(g.fparam + a), n, e - lo, [&](int j) { return dec(xv[j]); });
            bool gd = false;
            const float r = enc_fast(mu, gd);
            ng += gd;
            d = delta_p1_fast(r, a2v[e]);
            a2v[e] = r;
            a2v_vm[__ldg(F.vpos + e)] = r;
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

// Phase 1 and phase 2 of one iteration (or one RESIDUAL level).
void flood_phases(const DevGraph &g, const FloodPlanDev &P, float *a2v, float *a2v_vm, IterCtl ctl, cudaStream_t s)
{
    if (P.n_subs > 0) k_sub_products<<<(P.n_subs + P.sub_threads - 1) / P.sub_threads, P.sub_threads, 0, s>>>(g, P, a2v_vm);
    const int nb = P.nb_vars + P.nb_medium + (P.n_hub_rows + 7) / 8;
    if (nb > 0) k_beliefs<<<nb, 256, 0, s>>>(g, P, a2v_vm);
    if (P.n_wide > 0) k_wide_v2a<<<(P.n_wide + 255) / 256, 256, 0, s>>>(g, P, a2v);
    if (P.n_twarps > 0) k_a2v_lanes<<<(P.n_twarps + 7) / 8, 256, 0, s>>>(g, P, a2v, a2v_vm, ctl);
    if (P.n_warps > 0) k_a2v_fused<<<(P.n_warps + 7) / 8, 256, 0, s>>>(g, P, a2v, a2v_vm, ctl);
    if (P.n_wide > 0) k_a2v_wide<<<(P.n_wide + 255) / 256, 256, 0, s>>>(g, P, a2v, a2v_vm, ctl);
}

}  // namespace

void flood_sync(const DevGraph &g, const float *a2v, float *a2v_vm, cudaStream_t s)
{
    if (g.ne > 0) k_sync_vm<<<(g.ne + 255) / 256, 256, 0, s>>>(g, a2v, a2v_vm);
}

void flood_iteration(const DevGraph &g, const FloodPlanDev &F, float *a2v, float *a2v_vm, IterCtl ctl, float tol,
                     unsigned *hist, int *done, cudaStream_t s)
{
    FloodPlanDev P = F;
    P.done = done;
    flood_phases(g, P, a2v, a2v_vm, ctl, s);
    if (P.batch.n_graphs > 0) k_flood_batch_check<<<1, 1024, 0, s>>>(P.batch, done);
    else k_flood_check<<<1, kResSlots, 0, s>>>(ctl.res, hist, tol, done);
}

void flood_level(const DevGraph &g, const FloodPlanDev &F, float *a2v, float *a2v_vm, IterCtl ctl, int *done,
                 cudaStream_t s)
{
    FloodPlanDev P = F;
    P.done = done;
    flood_phases(g, P, a2v, a2v_vm, ctl, s);
}

void flood_check(IterCtl ctl, float tol, unsigned *hist, int *done, cudaStream_t s)
{
    k_flood_check<<<1, kResSlots, 0, s>>>(ctl.res, hist, tol, done);
}

cudaError_t flood_capture(const DevGraph &g, const FloodPlanDev &F, float *a2v, float *a2v_vm, IterCtl ctl, float tol,
                          unsigned *hist, int *done, int iters, cudaGraphExec_t *exec)
{
    cudaStream_t cap = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int k = 0; k < iters; ++k) flood_iteration(g, F, a2v, a2v_vm, ctl, tol, hist, done, cap);
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
    return (F.n_subs > 0) + (F.nb_vars + F.nb_medium + F.n_hub_rows > 0) + 2 * (F.n_wide > 0) + (F.n_twarps > 0) +
           (F.n_warps > 0) + 1;
}

}  // namespace fbp
