// CUDA kernels of the belief-propagation library (sm_103a).
//
// Message passing with local structure (Sec. 3.3, Sec. 4.3): every
// factor-to-variable message is a closed form in O(fan-in) of the incoming
// variable-to-factor messages, derived from the factor's logical meaning; the
// variable-to-factor messages are exclusion products (Eq. 1).
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
#include "fbp_internal.h"

#include <cmath>

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

// Factor-to-variable message of factor (type, p) with n variables to its
// variable at position i; getm(j) yields the incoming v->a message of position
// j scaled so that its larger entry is 1.
template <class GetM>
__device__ __forceinline__ P2 a2v_msg(int type, float p, int n, int i, GetM getm)
{
    if (type == kTypePRIOR) return P2{1.f - p, p};
    if (type == kTypeNOT) {
        P2 m = getm(1 - i);
        return P2{m.m1, m.m0};
    }
    if (type == kTypeEQ) {
        P2 acc{1.f, 1.f};
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            acc = mul(acc, getm(j));
            resc(acc);
        }
        return acc;
    }
    const int y = n - 1;
    float P1 = 1.f, P0 = 1.f, Ps = 1.f, D = 0.f, D0 = 0.f;
    for (int j = 0; j < y; ++j) {
        if (j == i) continue;
        P2 m = getm(j);
        float s = m.m0 + m.m1;
        D = fmaf(D, s, P1 * m.m0);
        D0 = fmaf(D0, s, P0 * m.m1);
        P1 *= m.m1;
        P0 *= m.m0;
        Ps *= s;
        if (Ps > 0x1p60f) {  // s in [1,2]: only long rows grow; scale all jointly
            P1 *= 0x1p-60f; P0 *= 0x1p-60f; Ps *= 0x1p-60f; D *= 0x1p-60f; D0 *= 0x1p-60f;
        }
    }
    const float q = 1.f - p;
    if (i == y) {
        switch (type) {
        case kTypeAND: return P2{D, P1};
        case kTypeOR: return P2{P0, D0};
        case kTypeNOISY_AND: return P2{fmaf(q, P1, D), p * P1};
        default: return P2{fmaf(q, P1, D), fmaf(p, P1, D)};  // NOISY_IMPLY
        }
    }
    P2 my = getm(y);
    float sy = my.m0 + my.m1;
    switch (type) {
    case kTypeAND: return P2{my.m0 * Ps, fmaf(my.m1, P1, my.m0 * D)};
    case kTypeOR: return P2{fmaf(my.m0, P0, my.m1 * D0), my.m1 * Ps};
    case kTypeNOISY_AND: return P2{my.m0 * Ps, fmaf(P1, fmaf(p, my.m1, q * my.m0), D * my.m0)};
    default: return P2{sy * Ps, fmaf(P1, fmaf(p, my.m1, q * my.m0), D * sy)};
    }
}

// Block-wide max of non-negative floats, one atomic per block into a slot.
__device__ __forceinline__ void block_max_to_slot(float v, IterCtl ctl)
{
    __shared__ unsigned s_max[32];
    unsigned bits = __float_as_uint(v);
    bits = __reduce_max_sync(0xffffffffu, bits);
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_max[warp] = bits;
    __syncthreads();
    if (warp == 0) {
        int nw = (blockDim.x + 31) >> 5;
        unsigned b = lane < nw ? s_max[lane] : 0u;
        b = __reduce_max_sync(0xffffffffu, b);
        if (lane == 0 && b) atomicMax(ctl.res + (blockIdx.x % kResSlots), b);
    }
}

// ---------------------------------------------------------------------------
// Phase 1, flooding: one thread per variable, two passes over its row.  The
// forward pass stores the prefix product (phi included) in each output slot;
// the backward pass multiplies in the suffix product.  Exclusion without
// division, so hard (0/1) messages stay exact.
// ---------------------------------------------------------------------------
__global__ void k_v2a_flood(const DevGraph g, const float *__restrict__ a2v,
                            float *__restrict__ v2a)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < g.nv; v += gridDim.x * blockDim.x) {
        const int lo = g.vptr[v], hi = g.vptr[v + 1];
        if (hi == lo) continue;
        P2 P = dec(g.phi[v]);
        for (int k = lo; k < hi; ++k) {
            const int e = g.vedge[k];
            v2a[e] = enc_z(P);
            P = mul(P, dec(a2v[e]));
            resc(P);
        }
        P2 S{1.f, 1.f};
        for (int k = hi - 1; k >= lo; --k) {
            const int e = g.vedge[k];
            P2 x = mul(dec_z(v2a[e]), S);
            bool gd = false;
            v2a[e] = enc(x, gd);
            S = mul(S, dec(a2v[e]));
            resc(S);
        }
    }
}

// ---------------------------------------------------------------------------
// Phase 2, flooding: one thread per factor, every outgoing message in place.
// ---------------------------------------------------------------------------
__global__ void k_a2v_flood(const DevGraph g, const float *__restrict__ v2a,
                            float *__restrict__ a2v, IterCtl ctl)
{
    float rmax = 0.f;
    unsigned long long ng = 0;
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < g.na; a += gridDim.x * blockDim.x) {
        const int lo = g.fptr[a], n = g.fptr[a + 1] - lo;
        const int type = g.ftype[a];
        const float p = g.fparam[a];
        auto getm = [&](int j) { return dec(v2a[lo + j]); };
        for (int i = 0; i < n; ++i) {
            P2 mu = a2v_msg(type, p, n, i, getm);
            bool gd = false;
            float r = enc(mu, gd);
            ng += gd;
            rmax = fmaxf(rmax, delta_p1(r, a2v[lo + i]));
            a2v[lo + i] = r;
        }
    }
    if (ng) atomicAdd(ctl.guards, ng);
    block_max_to_slot(rmax, ctl);
}

// ---------------------------------------------------------------------------
// One level of a static schedule: one thread per message (Sec. 4.3.1).
// ---------------------------------------------------------------------------
__global__ void k_level_edges(const DevGraph g, const int32_t *__restrict__ lev_edges, int32_t n,
                              int32_t level, const int32_t *__restrict__ vlev,
                              const float *__restrict__ cur, float *__restrict__ nxt, IterCtl ctl,
                              float *__restrict__ dres)
{
    float rmax = 0.f;
    unsigned long long ng = 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const int e = lev_edges[t];
        const int a = g.efac[e];
        const int lo = g.fptr[a], nf = g.fptr[a + 1] - lo, i = e - lo;
        auto getm = [&](int j) -> P2 {
            const int q = lo + j, vs = g.fvars[q];
            P2 m = dec(g.phi[vs]);
            for (int k = g.vptr[vs], kh = g.vptr[vs + 1]; k < kh; ++k) {
                const int ep = g.vedge[k];
                if (ep == q) continue;
                const float r = vlev[k] < level ? nxt[ep] : cur[ep];
                m = mul(m, dec(r));
                resc(m);
            }
            return norm_max(m);
        };
        P2 mu = a2v_msg(g.ftype[a], g.fparam[a], nf, i, getm);
        bool gd = false;
        float r = enc(mu, gd);
        ng += gd;
        const float d = delta_p1(r, cur[e]);
        rmax = fmaxf(rmax, d);
        nxt[e] = r;
        if (dres) dres[e] = d;
    }
    if (ng) atomicAdd(ctl.guards, ng);
    block_max_to_slot(rmax, ctl);
}

__global__ void k_marginals(const DevGraph g, const float *__restrict__ a2v, float *__restrict__ p1)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < g.nv; v += gridDim.x * blockDim.x) {
        P2 m = dec(g.phi[v]);
        for (int k = g.vptr[v], kh = g.vptr[v + 1]; k < kh; ++k) {
            m = mul(m, dec(a2v[g.vedge[k]]));
            resc(m);
        }
        float s = m.m0 + m.m1;
        p1[v] = (s > 0.f && isfinite(s)) ? __fdiv_rn(m.m1, s) : 0.5f;
    }
}

__global__ void k_decode_pairs(const float *__restrict__ rho, float *__restrict__ pairs, int32_t n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float p = p1_of(rho[i]);
        P2 m = dec(rho[i]);
        pairs[2 * i] = signbit(rho[i]) ? __fdiv_rn(1.f, 1.f + m.m1) : __fdiv_rn(m.m0, 1.f + m.m0);
        pairs[2 * i + 1] = p;
    }
}

__global__ void k_encode_pairs(const float *__restrict__ pairs, float *__restrict__ rho, int32_t n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        bool gd = false;
        rho[i] = enc(P2{pairs[2 * i], pairs[2 * i + 1]}, gd);
    }
}

__global__ void k_fill(float *x, float v, int32_t n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = v;
}

__global__ void k_copy_edges(const int32_t *__restrict__ edges, int32_t n, const float *__restrict__ src,
                             float *__restrict__ dst)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int e = edges[i];
        dst[e] = src[e];
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int num_sms()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

static inline int grid_for(int64_t n, int threads, int per_sm)
{
    int64_t need = (n + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms() * per_sm;
    if (need > cap) need = cap;
    return need < 1 ? 1 : (int)need;
}

void launch_v2a_flood(const DevGraph &g, const float *a2v, float *v2a, cudaStream_t s)
{
    if (g.nv == 0) return;
    k_v2a_flood<<<grid_for(g.nv, 256, 8), 256, 0, s>>>(g, a2v, v2a);
}

void launch_a2v_flood(const DevGraph &g, const float *v2a, float *a2v, IterCtl ctl, cudaStream_t s)
{
    if (g.na == 0) return;
    k_a2v_flood<<<grid_for(g.na, 256, 8), 256, 0, s>>>(g, v2a, a2v, ctl);
}

void launch_level(const DevGraph &g, const int32_t *lev_edges, int32_t n, int32_t level,
                  const int32_t *vlev, const float *cur, float *nxt, IterCtl ctl, float *dres,
                  cudaStream_t s)
{
    if (n == 0) return;
    k_level_edges<<<grid_for(n, 128, 16), 128, 0, s>>>(g, lev_edges, n, level, vlev, cur, nxt, ctl, dres);
}

void launch_marginals(const DevGraph &g, const float *a2v, float *p1, cudaStream_t s)
{
    if (g.nv == 0) return;
    k_marginals<<<grid_for(g.nv, 256, 8), 256, 0, s>>>(g, a2v, p1);
}

void launch_decode_pairs(const float *rho, float *pairs, int32_t n, cudaStream_t s)
{
    if (n == 0) return;
    k_decode_pairs<<<grid_for(n, 256, 8), 256, 0, s>>>(rho, pairs, n);
}

void launch_encode_pairs(const float *pairs, float *rho, int32_t n, cudaStream_t s)
{
    if (n == 0) return;
    k_encode_pairs<<<grid_for(n, 256, 8), 256, 0, s>>>(pairs, rho, n);
}

void launch_fill(float *x, float v, int32_t n, cudaStream_t s)
{
    if (n == 0) return;
    k_fill<<<grid_for(n, 256, 8), 256, 0, s>>>(x, v, n);
}

void launch_copy_edges(const int32_t *edges, int32_t n, const float *src, float *dst, cudaStream_t s)
{
    if (n == 0) return;
    k_copy_edges<<<grid_for(n, 256, 8), 256, 0, s>>>(edges, n, src, dst);
}

}  // namespace fbp
