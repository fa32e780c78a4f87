// Device-side schedule of the RESIDUAL strategy (the reading of the residual
// strategy: iteration t >= 2 ranks each factor by the largest |dP(x=1)| of
// iteration t-1's writes into its variables, classes >= 1e-2, [1e-4, 1e-2),
// [tol, 1e-4), factors below tol skipped; Algorithm 2 over the active edges).
//
// With at most three classes, Algorithm 2 (Sec. 4.2.3) cuts at most once per
// class: edges of one class never depend on each other (equal ranks), so a
// class-c edge ends the current level only if it reads a message written by
// an edge of a lower class in that level -- and after such a cut the level
// holds class c alone.  The scan therefore reduces to, per class c = 1, 2:
//   NextSet = the lower-class edges of the current level,
//   cut_c   = the first class-c edge (in edge order) e = (a, v) such that some
//             other variable u of a receives an edge of NextSet,
// and a level index per edge from the cuts.  Each step is a data-parallel
// pass (per-variable counts, per-factor tests, a min over edges), so a
// RESIDUAL iteration of a million-edge graph needs no host round trip of its
// edges.
#include "fbp_msg.cuh"
#include "fbp_residual.h"

#include <climits>

namespace fbp {

namespace {

// vres[u] = largest |dP| of the previous iteration's writes into u: one
// thread per edge (hub variables have 1e5 incident edges), the maximum taken
// on the float bits (non-negative values order like their bits).
__global__ void k_rs_vres(const DevGraph g, const float *__restrict__ dres, unsigned *__restrict__ vres)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= g.ne) return;
    const unsigned bits = __float_as_uint(__ldg(dres + e));
    if (bits) max_bits(vres + __ldg(g.fvars + e), bits);
}

// Class of every factor from the largest change at its variables; counts the
// active edges into ctl[kRsActive].
__global__ void k_rs_class(const DevGraph g, const unsigned *__restrict__ vres, double tol,
                           int8_t *__restrict__ fcls, int *ctl)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    int active = 0;
    if (a < g.na) {
        const int lo = __ldg(g.fptr + a), hi = __ldg(g.fptr + a + 1);
        float rho = 0.f;
        for (int q = lo; q < hi; ++q) rho = fmaxf(rho, __uint_as_float(__ldg(vres + __ldg(g.fvars + q))));
        const double r = rho;
        const int c = r >= 1e-2 ? 0 : r >= 1e-4 ? 1 : r >= tol ? 2 : -1;
        fcls[a] = (int8_t)c;
        if (c >= 0) active = hi - lo;
    }
    active = __reduce_add_sync(0xffffffffu, active);
    if ((threadIdx.x & 31) == 0 && active) atomicAdd(ctl + kRsActive, active);
}

// NextSet membership of edge e when the scan reaches class c: an edge of a
// lower class in the current level.  For c = 1 that is every class-0 edge;
// for c = 2 the class-1 edges from cut_1 on, or (without a cut at class 1)
// every class-0 and class-1 edge.
__device__ __forceinline__ bool in_next(int ce, int e, int c, int cut1)
{
    if (c == 1) return ce == 0;
    if (cut1 != INT_MAX) return ce == 1 && e >= cut1;
    return ce == 0 || ce == 1;
}

// cnt[u] = 1 if some edge of NextSet enters variable u (class c of the
// scan), from one thread per edge (all writers store the same 1).
__global__ void k_rs_count(const DevGraph g, const int8_t *__restrict__ fcls, int c, const int *ctl,
                           int *__restrict__ cnt)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= g.ne) return;
    if (in_next(fcls[__ldg(g.efac + e)], e, c, ctl[kRsCut1])) cnt[__ldg(g.fvars + e)] = 1;
}

// cut_c: the first class-c edge (a, v) such that another variable of a
// receives a NextSet edge.  (a's own edges are class c, never in NextSet.)
__global__ void k_rs_cut(const DevGraph g, const int8_t *__restrict__ fcls, int c, const int *__restrict__ cnt,
                         int *ctl)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    int first = INT_MAX;
    if (a < g.na && fcls[a] == c) {
        const int lo = __ldg(g.fptr + a), hi = __ldg(g.fptr + a + 1);
        int k = 0;  // variables of a that receive a NextSet edge
        for (int q = lo; q < hi; ++q) k += cnt[__ldg(g.fvars + q)] > 0;
        for (int q = lo; q < hi && first == INT_MAX; ++q)
            if (k - (cnt[__ldg(g.fvars + q)] > 0) > 0) first = q;
    }
    first = __reduce_min_sync(0xffffffffu, first);
    if ((threadIdx.x & 31) == 0 && first != INT_MAX) atomicMin(ctl + (c == 1 ? kRsCut1 : kRsCut2), first);
}

// Level of every edge (-1: skipped this iteration).
__global__ void k_rs_level(const DevGraph g, const int8_t *__restrict__ fcls, const int *ctl,
                           int8_t *__restrict__ elev)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= g.ne) return;
    const int c = fcls[__ldg(g.efac + e)];
    const int cut1 = ctl[kRsCut1], cut2 = ctl[kRsCut2];
    const int base2 = cut1 != INT_MAX;  // the level at which class 2 starts
    int lv = -1;
    if (c == 0) lv = 0;
    else if (c == 1) lv = (cut1 != INT_MAX && e >= cut1) ? 1 : 0;
    else if (c == 2) lv = base2 + ((cut2 != INT_MAX && e >= cut2) ? 1 : 0);
    elev[e] = (int8_t)lv;
}

__global__ void k_rs_reset(int *ctl)
{
    ctl[kRsActive] = 0;
    ctl[kRsCut1] = INT_MAX;
    ctl[kRsCut2] = INT_MAX;
}

}  // namespace

void residual_schedule(const DevGraph &g, const float *dres, double tol, ResidualWork &w, cudaStream_t s)
{
    const int tb = 256;
    k_rs_reset<<<1, 1, 0, s>>>(w.ctl);
    cudaMemsetAsync(w.vres, 0, sizeof(unsigned) * (size_t)g.nv, s);
    if (g.ne > 0) k_rs_vres<<<(g.ne + tb - 1) / tb, tb, 0, s>>>(g, dres, w.vres);
    if (g.na > 0) k_rs_class<<<(g.na + tb - 1) / tb, tb, 0, s>>>(g, w.vres, tol, w.fcls, w.ctl);
    for (int c = 1; c <= 2; ++c) {
        cudaMemsetAsync(w.cnt, 0, sizeof(int) * (size_t)g.nv, s);
        if (g.ne > 0) k_rs_count<<<(g.ne + tb - 1) / tb, tb, 0, s>>>(g, w.fcls, c, w.ctl, w.cnt);
        if (g.na > 0) k_rs_cut<<<(g.na + tb - 1) / tb, tb, 0, s>>>(g, w.fcls, c, w.cnt, w.ctl);
    }
    if (g.ne > 0) k_rs_level<<<(g.ne + tb - 1) / tb, tb, 0, s>>>(g, w.fcls, w.ctl, w.elev);
}

}  // namespace fbp
