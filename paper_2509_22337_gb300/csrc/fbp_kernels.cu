// CUDA kernels of the belief-propagation library (sm_103a): marginals
// (Eq. 3), message (de)serialisation and fills.  The message algebra and the
// closed forms live in fbp_msg.cuh; flooding in fbp_flood.cu; static
// schedules in the persistent engine (fbp_engine.cu).
#include "fbp_msg.cuh"

#include <cmath>

namespace fbp {

// Marginals (Eq. 3): P(x_v = 1) from phi_v times every incoming a->v message.
// Rows of at most kMargRowMax entries: one thread each, the entries in row
// order (loaded kMargLoads at a time, multiplied in order).  Longer rows are
// left to k_marginals_long.
constexpr int kMargRowMax = 256;
constexpr int kMargLoads = 16;

__global__ void k_marginals(const DevGraph g, const float *__restrict__ a2v, float *__restrict__ p1)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < g.nv; v += gridDim.x * blockDim.x) {
        const int lo = g.vptr[v], hi = g.vptr[v + 1];
        if (hi - lo > kMargRowMax) continue;
        P2 m = dec(g.phi[v]);
        for (int k0 = lo; k0 < hi; k0 += kMargLoads) {
            float r[kMargLoads];
#pragma unroll
            for (int u = 0; u < kMargLoads; ++u) r[u] = k0 + u < hi ? a2v[g.vedge[k0 + u]] : 1.f;
#pragma unroll
            for (int u = 0; u < kMargLoads; ++u)
                if (k0 + u < hi) {
                    m = mul(m, dec(r[u]));
                    resc(m);
                }
        }
        float s = m.m0 + m.m1;
        p1[v] = (s > 0.f && isfinite(s)) ? __fdiv_rn(m.m1, s) : 0.5f;
    }
}

// Marginals of the rows longer than kMargRowMax, one block of 256 threads per
// row: entry k goes to slot (k - row start) mod 256, each slot multiplies its
// entries in order, the slots are combined by an xor butterfly (j with
// j^128, then j^64, ..., j^1), and phi_v is multiplied in last.  A grouping
// of its own, fixed whatever launches it.
__global__ void __launch_bounds__(256) k_marginals_long(const DevGraph g, const float *__restrict__ a2v,
                                                        float *__restrict__ p1, const int32_t *__restrict__ rows)
{
    constexpr int kB = 8;  // entries per thread whose loads are in flight together
    __shared__ P2 s_m[256];
    const int v = rows[blockIdx.x], j = threadIdx.x;
    const int lo = g.vptr[v], hi = g.vptr[v + 1];
    P2 m{1.f, 1.f};
    for (int k0 = lo + j; k0 < hi; k0 += 256 * kB) {
        float r[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u) r[u] = k0 + 256 * u < hi ? a2v[g.vedge[k0 + 256 * u]] : 1.f;
#pragma unroll
        for (int u = 0; u < kB; ++u)
            if (k0 + 256 * u < hi) {
                m = mul(m, dec(r[u]));
                resc(m);
            }
    }
    for (int o = 128; o >= 32; o >>= 1) {
        s_m[j] = m;
        __syncthreads();
        if (j < o) {
            m = mul(m, s_m[j + o]);
            resc(m);
        }
        __syncthreads();
    }
    if (j >= 32) return;
    for (int o = 16; o > 0; o >>= 1) {
        const P2 t{__shfl_xor_sync(0xffffffffu, m.m0, o), __shfl_xor_sync(0xffffffffu, m.m1, o)};
        m = mul(m, t);
        resc(m);
    }
    if (j == 0) {
        m = mul(dec(g.phi[v]), m);
        resc(m);
        const float s = m.m0 + m.m1;
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

void launch_marginals_long(const DevGraph &g, const float *a2v, float *p1, const int32_t *rows, int32_t n,
                           cudaStream_t s)
{
    if (n > 0) k_marginals_long<<<n, 256, 0, s>>>(g, a2v, p1, rows);
}

int marginals_row_max() { return kMargRowMax; }

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
