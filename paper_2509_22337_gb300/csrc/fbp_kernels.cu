// CUDA kernels of the belief-propagation library (sm_103a): marginals
// (Eq. 3), message (de)serialisation and fills.  The message algebra and the
// closed forms live in fbp_msg.cuh; flooding in fbp_flood.cu; static
// schedules in the persistent engine (fbp_engine.cu).
#include "fbp_msg.cuh"

#include <cmath>

namespace fbp {

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
