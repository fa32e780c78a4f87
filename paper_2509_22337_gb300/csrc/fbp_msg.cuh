// Device-side message algebra shared by the CUDA kernels of the library:
// the one-float message encoding (see fbp_internal.h), products with joint
// power-of-two rescaling, and the closed-form factor-to-variable messages of
// the logical factor types (Sec. 3.3's local structure).
//
// Closed forms (premises x_1..x_n, output y; incoming m_j = (m_j0, m_j1),
// s_j = m_j0 + m_j1; products over premises other than the target):
//   P1 = prod m_j1, P0 = prod m_j0, Ps = prod s_j,
//   D  = Ps - P1 = sum_k (prod_{j<k} m_j1) m_k0 (prod_{j>k} s_j)   (no cancellation)
//   D0 = Ps - P0 = sum_k (prod_{j<k} m_j0) m_k1 (prod_{j>k} s_j)
//   type          to y                          to premise x_i
//   AND           (D, P1)                       (y0 Ps, y1 P1 + y0 D)
//   OR            (P0, D0)                      (y0 P0 + y1 D0, y1 Ps)
//   NOT           (x1, x0)                      (y1, y0)
//   EQ            (prod m_u0, prod m_u1) over all other variables
//   NOISY_AND(p)  ((1-p)P1 + D, p P1)           (y0 Ps, P1 (p y1 + (1-p) y0) + D y0)
//   NOISY_IMPLY(p)((1-p)P1 + D, p P1 + D)       (sy Ps, P1 (p y1 + (1-p) y0) + D sy)
//   PRIOR(p)      (1-p, p)
// Each is the sum over the factor's sub-messages (Eq. 4) with the common
// products factored out, so it equals Algorithm 1 on the factor's term list.
#pragma once

#include "fbp_internal.h"

namespace fbp {

struct P2 {
    float m0, m1;
};

__device__ __forceinline__ P2 dec(float r)
{
    return signbit(r) ? P2{1.f, -r} : P2{r, 1.f};
}

// (0,0) is stored as NaN inside a pass (prefix products only).
__device__ __forceinline__ P2 dec_z(float r)
{
    return isnan(r) ? P2{0.f, 0.f} : dec(r);
}

__device__ __forceinline__ float enc_z(P2 m)
{
    if (m.m0 == 0.f && m.m1 == 0.f) return __int_as_float(0x7fc00000);
    return (m.m1 >= m.m0) ? __fdiv_rn(m.m0, m.m1) : -__fdiv_rn(m.m1, m.m0);
}

// Normalise to the larger entry; zero mass (or a non-finite sum) becomes the
// uniform message and raises `guard`.
__device__ __forceinline__ float enc(P2 m, bool &guard)
{
    float s = m.m0 + m.m1;
    if (!(s > 0.f) || !isfinite(s)) {
        guard = true;
        return 1.f;
    }
    return (m.m1 >= m.m0) ? __fdiv_rn(m.m0, m.m1) : -__fdiv_rn(m.m1, m.m0);
}

// P(x = 1) of a rho-encoded message.
__device__ __forceinline__ float p1_of(float r)
{
    return signbit(r) ? __fdiv_rn(-r, 1.f - r) : __fdiv_rn(1.f, 1.f + r);
}

// |P(x=1 | new) - P(x=1 | old)| without cancellation.  With m1 the larger
// entry (rho >= 0) P = 1/(1+rho); with m0 the larger, P = |rho|/(1+|rho|).
// Same orientation: the difference is |rho_o - rho_n| / ((1+|rho_n|)(1+|rho_o|)),
// exact up to a few ulps of the result.  Opposite orientation: the two
// probabilities lie on either side of 1/2, and the distance is the sum of
// their distances to 1/2, (1-|rho|)/(2(1+|rho|)) each.
__device__ __forceinline__ float delta_p1(float rn, float ro)
{
    const float an = fabsf(rn), ao = fabsf(ro);
    if (signbit(rn) == signbit(ro)) return __fdiv_rn(fabsf(ao - an), (1.f + an) * (1.f + ao));
    return __fdiv_rn(1.f - an, 2.f * (1.f + an)) + __fdiv_rn(1.f - ao, 2.f * (1.f + ao));
}

__device__ __forceinline__ P2 mul(P2 a, P2 b) { return P2{a.m0 * b.m0, a.m1 * b.m1}; }

// Joint power-of-two rescale: leaves the normalised message unchanged.
__device__ __forceinline__ void resc(P2 &a)
{
    float mx = fmaxf(a.m0, a.m1);
    if (mx < 0x1p-60f && mx > 0.f) {
        a.m0 *= 0x1p60f;
        a.m1 *= 0x1p60f;
    }
}

// Scale so that the larger entry is 1; zero mass -> uniform (guard).
__device__ __forceinline__ P2 norm_max(P2 m)
{
    float mx = fmaxf(m.m0, m.m1);
    if (!(mx > 0.f) || !isfinite(mx)) return P2{1.f, 1.f};
    float inv = __frcp_rn(mx);
    return P2{m.m0 == mx ? 1.f : m.m0 * inv, m.m1 == mx ? 1.f : m.m1 * inv};
}

// Products over a factor's premises other than the target (see the closed
// forms above), accumulated in premise order.  A message enters scaled so
// that its larger entry is 1; the sums s_j lie in [1, 2], so only Ps can grow,
// and all five are scaled down together by 2^-60 past 2^60 (the message is
// homogeneous in them).
struct Acc5 {
    float P1 = 1.f, P0 = 1.f, Ps = 1.f, D = 0.f, D0 = 0.f;
};

__device__ __forceinline__ void acc5_add(Acc5 &a, P2 m)
{
    const float s = m.m0 + m.m1;
    a.D = fmaf(a.D, s, a.P1 * m.m0);
    a.D0 = fmaf(a.D0, s, a.P0 * m.m1);
    a.P1 *= m.m1;
    a.P0 *= m.m0;
    a.Ps *= s;
    if (a.Ps > 0x1p60f) {
        a.P1 *= 0x1p-60f; a.P0 *= 0x1p-60f; a.Ps *= 0x1p-60f; a.D *= 0x1p-60f; a.D0 *= 0x1p-60f;
    }
}

// The message of factor (type, p) to its output (to_output) or to a premise,
// from the products over the other premises and the output's incoming message
// my (unused for the output).  Every type's message is a combination of the
// five products with coefficients selected per type, so a warp that holds
// factors of different types runs one instruction stream:
//   target = output:   mu0 = a0 P1 + a1 D + a2 P0,   mu1 = b0 P1 + b1 D + b2 D0 + b3 P0
//   target = premise:  mu0 = c0 Ps + c1 P0 + c2 D0,  mu1 = d0 P1 + d1 D + d2 Ps
// (NOT reads its single premise through P1/P0; EQ treats the last variable
// like the output; PRIOR has no premises, so P1 = P0 = 1 and D = D0 = 0.)
__device__ __forceinline__ P2 a2v_finish(int type, float p, bool to_output, const Acc5 &A, P2 my)
{
    const unsigned t = 1u << type;
    constexpr unsigned AND = 1u << kTypeAND, OR = 1u << kTypeOR, NOT = 1u << kTypeNOT, EQ = 1u << kTypeEQ,
                       NI = 1u << kTypeNOISY_IMPLY, NA = 1u << kTypeNOISY_AND, PR = 1u << kTypePRIOR;
    const float q = 1.f - p;
    if (to_output) {
        const float a0 = (t & NOT) ? 1.f : (t & (NA | NI | PR)) ? q : 0.f;
        const float a1 = (t & (AND | NA | NI)) ? 1.f : 0.f;
        const float a2 = (t & (OR | EQ)) ? 1.f : 0.f;
        const float b0 = (t & (AND | EQ)) ? 1.f : (t & (NA | NI | PR)) ? p : 0.f;
        const float b1 = (t & NI) ? 1.f : 0.f;
        const float b2 = (t & OR) ? 1.f : 0.f;
        const float b3 = (t & NOT) ? 1.f : 0.f;
        return P2{fmaf(a0, A.P1, fmaf(a1, A.D, a2 * A.P0)), fmaf(b0, A.P1, fmaf(b1, A.D, fmaf(b2, A.D0, b3 * A.P0)))};
    }
    const float sy = my.m0 + my.m1, w = fmaf(p, my.m1, q * my.m0);
    const float c0 = (t & (AND | NA)) ? my.m0 : (t & NOT) ? my.m1 : (t & NI) ? sy : 0.f;
    const float c1 = (t & (OR | EQ)) ? my.m0 : 0.f;
    const float c2 = (t & OR) ? my.m1 : 0.f;
    const float d0 = (t & (AND | EQ)) ? my.m1 : (t & (NA | NI)) ? w : 0.f;
    const float d1 = (t & (AND | NA)) ? my.m0 : (t & NI) ? sy : 0.f;
    const float d2 = (t & OR) ? my.m1 : (t & NOT) ? my.m0 : 0.f;
    return P2{fmaf(c0, A.Ps, fmaf(c1, A.P0, c2 * A.D0)), fmaf(d0, A.P1, fmaf(d1, A.D, d2 * A.Ps))};
}

// Factor-to-variable message of factor (type, p) with n variables to its
// variable at position i; getm(j) yields the incoming v->a message of position
// j scaled so that its larger entry is 1.
template <class GetM>
__device__ __forceinline__ P2 a2v_unified(int type, float p, int n, int i, GetM getm)
{
    const int y = n - 1;
    Acc5 A;
    for (int j = 0; j < y; ++j) {
        if (j == i) continue;
        acc5_add(A, getm(j));
    }
    if (i == y) return a2v_finish(type, p, true, A, P2{1.f, 1.f});
    return a2v_finish(type, p, false, A, getm(y));
}

// Algorithm 1 for a generic factor a with n variables, target position i:
// each term that does not conflict with the target's value adds its weight
// times, for every other variable, the incoming message at the term's value
// (the sum of both entries where the term leaves the variable free).  getm(j)
// yields position j's v->a message scaled so that its larger entry is 1.
template <class GetM>
__device__ __forceinline__ P2 a2v_terms(const DevGraph &g, int a, int n, int i, GetM getm)
{
    const int t0 = __ldg(g.tptr + a), t1 = __ldg(g.tptr + a + 1);
    const int8_t *ind = g.tind + __ldg(g.tioff + a);
    P2 mu{0.f, 0.f};
    for (int t = t0; t < t1; ++t, ind += n) {
        float prod = __ldg(g.tw + t);
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            const P2 m = getm(j);
            const int c = __ldg(ind + j);
            prod *= c < 0 ? m.m0 + m.m1 : (c ? m.m1 : m.m0);
        }
        const int ci = __ldg(ind + i);
        if (ci <= 0) mu.m0 += prod;  // free (-1) or 0: counts toward x_i = 0
        if (ci != 0) mu.m1 += prod;  // free (-1) or 1: counts toward x_i = 1
    }
    return mu;
}

// Hardware reciprocal approximation with subnormals flushed
// (rcp.approx.ftz.f32: relative error within a couple of ulp).  Callers pass
// arguments whose reciprocal is normal as well, where it is the same
// approximation as the subnormal-keeping form, at a fraction of its cost.
__device__ __forceinline__ float rcp_normal(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Encoding through the reciprocal of the larger entry (result within a few
// ulp of the quotient, clamped to |rho| <= 1); zero mass -> uniform.  A larger
// entry outside [2^-64, 2^64] is first brought inside by a power of two,
// applied to both entries (exact unless the smaller one then leaves the
// normal range, where the quotient itself is below it).
__device__ __forceinline__ float enc_fast(P2 m, bool &guard)
{
    const float s = m.m0 + m.m1;
    if (!(s > 0.f) || !isfinite(s)) {
        guard = true;
        return 1.f;
    }
    float mx = fmaxf(m.m0, m.m1), mn = fminf(m.m0, m.m1);
    if (!(mx >= 0x1p-64f && mx <= 0x1p64f)) {
        const float k = mx < 1.f ? 0x1p64f : 0x1p-64f;
        mx *= k;
        mn *= k;
    }
    const float r = fminf(mn * rcp_normal(mx), 1.f);
    return m.m1 >= m.m0 ? r : -r;
}

// delta_p1 for the convergence test only: approximate reciprocals (a few
// ulp) of arguments in [1, 4].
__device__ __forceinline__ float delta_p1_fast(float rn, float ro)
{
    const float an = fabsf(rn), ao = fabsf(ro);
    if (signbit(rn) == signbit(ro)) return fabsf(ao - an) * rcp_normal((1.f + an) * (1.f + ao));
    return (1.f - an) * rcp_normal(2.f * (1.f + an)) + (1.f - ao) * rcp_normal(2.f * (1.f + ao));
}

// Raise a max word to `bits` (the bits of a non-negative float, so that the
// integer and float orders agree).  The word only grows while it collects a
// maximum, so a read that already shows at least `bits` makes the atomic
// unnecessary; this keeps thousands of blocks from serialising on one word.
__device__ __forceinline__ void max_bits(unsigned *word, unsigned bits)
{
    if (bits > __ldcg(word)) atomicMax(word, bits);
}

// Warp max of a non-negative float, then block max via shared memory; the
// result is valid in thread 0.  Every thread of the block must call it.
__device__ __forceinline__ float block_max(float v)
{
    __shared__ unsigned s_max[32];
    unsigned bits = __reduce_max_sync(0xffffffffu, __float_as_uint(v));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s_max[warp] = bits;
    __syncthreads();
    unsigned b = 0;
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        b = lane < nw ? s_max[lane] : 0u;
        b = __reduce_max_sync(0xffffffffu, b);
    }
    return __uint_as_float(b);
}

}  // namespace fbp
