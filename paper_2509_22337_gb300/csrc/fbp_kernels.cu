// CUDA kernels of the belief-propagation library (sm_103a): the flooding
// (PARALL) phases, marginals (Eq. 3) and message (de)serialisation.  The
// message algebra and the closed forms live in fbp_msg.cuh.
#include "fbp_msg.cuh"

#include <cmath>

namespace fbp {

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
            P2 mu = a2v_unified(type, p, n, i, getm);
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

}  // namespace fbp
