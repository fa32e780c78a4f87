// fbp_run_fixed_scratch (include/fbp_fixed.h): the persistent level engine of
// fbp_run with its per-run scratch taken from one static device array, so
// that the call allocates no device memory at all.
//
// Callers that cannot allocate while running -- a serving loop whose device
// memory is all committed to resident graphs before the first request, or a
// latency-bound caller that cannot take an allocation (and the device
// synchronisation it may bring) inside a request -- get the same run as
// fbp_run without the on-demand growth of the per-iteration residual words.
#include "fbp.h"
#include "fbp_fixed.h"
#include "fbp_graph_impl.h"
#include "fbp_internal.h"

#include <cstring>
#include <mutex>

using namespace fbp;

namespace {

// Scratch layout (byte offsets).  Every word below must be zero when the
// engine kernel starts; the entry point clears them on the graph's stream
// before each launch.
constexpr size_t kBarOff = 0;      // unsigned[2]: grid-barrier counter, generation
constexpr size_t kOutOff = 16;     // int32[4]: iterations, status, error word, spare
constexpr size_t kGuardOff = 32;   // unsigned long long: zero-mass guards taken
constexpr size_t kResOff = 256;    // unsigned[FBP_FIXED_SCRATCH_MAX_ITERS]: residual bits
static_assert(kResOff + 4 * (size_t)FBP_FIXED_SCRATCH_MAX_ITERS == FBP_FIXED_SCRATCH_BYTES,
              "scratch layout and FBP_FIXED_SCRATCH_BYTES disagree");

static __device__ __align__(256) unsigned char fbp_fixed_scratch[FBP_FIXED_SCRATCH_BYTES];

// Device address of fbp_fixed_scratch, looked up once per device (with that
// device current) and kept.
constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
unsigned char *g_addr[kMaxDevices] = {};

#define FIXED_CUDA_TRY(call)                                                                 \
    do {                                                                                     \
        cudaError_t _e = (call);                                                             \
        if (_e != cudaSuccess)                                                               \
            return fail(FBP_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(_e));       \
    } while (0)

int scratch_address(unsigned char **out)
{
    int dev = -1;
    FIXED_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices)
        return fail(FBP_ERR_CUDA, "device %d is beyond the %d devices the fixed scratch tracks", dev,
                    kMaxDevices);
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, fbp_fixed_scratch);
        if (e != cudaSuccess || !p)
            return fail(FBP_ERR_CUDA, "cudaGetSymbolAddress(fbp_fixed_scratch) on device %d failed: %s", dev,
                        cudaGetErrorString(e));
        g_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_addr[dev];
    return FBP_OK;
}

}  // namespace

extern "C" int fbp_run_fixed_scratch(fbp_graph *g, int32_t max_iters, double tol, int32_t *iters_out,
                                     double *residual_out)
{
    clear_error();  // fbp_last_error reports this call only
    if (!g) return fail(FBP_ERR_INVALID_ARG, "graph is NULL");
    if (max_iters < 0 || !(tol >= 0.0)) return fail(FBP_ERR_INVALID_ARG, "bad argument");
    if (max_iters > FBP_FIXED_SCRATCH_MAX_ITERS)
        return fail(FBP_ERR_INVALID_ARG,
                    "max_iters %d exceeds the fixed scratch limit of %d iterations (FBP_FIXED_SCRATCH_MAX_ITERS)",
                    max_iters, FBP_FIXED_SCRATCH_MAX_ITERS);
    if (g->strategy == FBP_PARALL || g->strategy == FBP_RESIDUAL)
        return fail(FBP_ERR_INVALID_ARG, "fbp_run_fixed_scratch needs a static strategy "
                                         "(SEQFIX, TOPO, TOPO_FB or CUSTOM_RANK)");
    if (g->terms_needed && !g->terms_set)
        return fail(FBP_ERR_INVALID_ARG, "generic (FBP_TERMS) factors have no terms: call fbp_set_factor_terms");
    unsigned char *base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    unsigned *bar = reinterpret_cast<unsigned *>(base + kBarOff);
    int32_t *out = reinterpret_cast<int32_t *>(base + kOutOff);
    unsigned long long *guards = reinterpret_cast<unsigned long long *>(base + kGuardOff);
    unsigned *res = reinterpret_cast<unsigned *>(base + kResOff);

    const HostCSR &h = g->h;
    g->stats = fbp_stats{};
    for (auto &ls : g->halves) g->stats.levels += (int32_t)ls.lp.size() - 1;
    FIXED_CUDA_TRY(cudaMemsetAsync(base, 0, kResOff, g->stream));
    FIXED_CUDA_TRY(cudaMemsetAsync(res, 0, sizeof(unsigned) * (size_t)(max_iters > 0 ? max_iters : 1), g->stream));
    FIXED_CUDA_TRY(cudaEventRecord(g->ev0, g->stream));

    int32_t it = 0;
    unsigned res_bits = 0;
    int status = FBP_NOT_CONVERGED;
    if (max_iters > 0) {
        // always the persistent engine in one launch (the per-level launches
        // of FBP_OPT_ENGINE=0 would compute the same messages)
        EngineArgs A = engine_args(g);
        A.guards = guards;
        A.bar = bar;
        A.out = out;
        A.res = res;
        A.max_iters = max_iters;
        A.tol = (float)tol;
        int grid = 1, cluster = 0;
        engine_shape(g, &grid, &cluster);
        FIXED_CUDA_TRY(launch_engine(A, grid, cluster, g->stream));
        g->stats.kernel_launches += 1;
        int32_t o[4] = {0, 0, 0, 0};
        FIXED_CUDA_TRY(cudaMemcpyAsync(o, out, sizeof o, cudaMemcpyDeviceToHost, g->stream));
        FIXED_CUDA_TRY(cudaStreamSynchronize(g->stream));
        if (o[2])
            return fail(FBP_ERR_TIMEOUT, "a device-side barrier wait expired (spin limit %lld cycles)",
                        (long long)g->spin_limit);
        it = o[0];
        status = o[1] == 0 ? FBP_OK : FBP_NOT_CONVERGED;
        g->cur ^= (it * A.n_halves) & 1;
        g->stats.updates += (int64_t)it * A.n_halves * h.ne;
        if (it >= 1)
            FIXED_CUDA_TRY(cudaMemcpyAsync(&res_bits, res + (it - 1), sizeof res_bits, cudaMemcpyDeviceToHost,
                                           g->stream));
    }
    FIXED_CUDA_TRY(cudaEventRecord(g->ev1, g->stream));
    unsigned long long n_guards = 0;
    FIXED_CUDA_TRY(cudaMemcpyAsync(&n_guards, guards, sizeof n_guards, cudaMemcpyDeviceToHost, g->stream));
    FIXED_CUDA_TRY(cudaEventSynchronize(g->ev1));
    FIXED_CUDA_TRY(cudaStreamSynchronize(g->stream));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, g->ev0, g->ev1);
    float r;
    std::memcpy(&r, &res_bits, sizeof r);
    g->stats.iters = it;
    g->stats.residual = (double)r;
    g->stats.run_ms = ms;
    g->stats.guards = (int64_t)n_guards;
    if (iters_out) *iters_out = it;
    if (residual_out) *residual_out = (double)r;
    return status;
}
