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
//   longer rows               one thread per 32-entry sub-chunk (in the same
//                             launch as the short rows); then a row of 2..8
//                             sub-chunks (at most FBP_OPT_FLOOD_HUB_MIN
//                             entries) combined by one thread, a longer one
//                             by one block of 256 threads
// The product of every row longer than 8 entries is grouped one way only,
// whichever kernel carries the row: the row is cut into 32-entry sub-chunks,
// each multiplied in order; sub-chunk s goes to slot s mod 256 (a slot
// multiplies its sub-chunks in order), and the 256 slots are combined by an
// xor butterfly (slot j with slot j^128, then j^64, ..., j^2, j^1).  A row of
// at most 256 entries fills slots 0..7 only, and the one-thread combine
// evaluates exactly that butterfly (a product with an empty slot is the value
// itself), so the thread and the block combines compute the same bits and
// the split options (FBP_OPT_FLOOD_HUB_MIN, _CHUNK) only move work between
// kernels.  phi_v is multiplied in last.  Every multiply rounds the exact
// product once (the mantissa/exponent form never goes subnormal), so only
// this grouping decides the result.
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
#include "fbp_flood_dev.cuh"

namespace fbp {

namespace {

using namespace fdev;

// ----------------------------------------------------------------------------
// Phase 1
// ----------------------------------------------------------------------------
__global__ void k_sync_vm(const DevGraph g, const float *__restrict__ a2v, float *__restrict__ a2v_vm)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < g.ne) a2v_vm[k] = a2v[__ldg(g.vedge + k)];
}

// Phase 1, first pass (two roles that share no data, so the long per-thread
// product chains of the sub-chunks overlap with the short rows' loads).
// Blocks [0, nb_subs): the products of the 32-entry sub-chunks of the rows
// longer than 8 entries, sub_threads per block, one thread per sub-chunk (a
// row of one sub-chunk gets its belief here).  The nb_vars blocks from
// nb_subs on: the belief of every variable of degree <= 8, one thread per
// variable, each thread taking variables a grid of those blocks apart.
__global__ void __launch_bounds__(256, 8) k_beliefs(const DevGraph g, FloodPlanDev F, const float *__restrict__ a2v_vm)
{
    if (*(volatile const int *)F.done) return;
    const int nb_subs = (F.n_subs + F.sub_threads - 1) / F.sub_threads;
    const int b = blockIdx.x;
    if (b < nb_subs) {
        const int k = b * F.sub_threads + threadIdx.x;
        if (threadIdx.x < F.sub_threads && k < F.n_subs) sub_product_item<false>(g, F, a2v_vm, k);
        return;
    }
    belief_var_loop(g, F, a2v_vm, (b - nb_subs) * blockDim.x + threadIdx.x, F.nb_vars * blockDim.x);
}

// Phase 1, second pass: the rows of several sub-chunks combine their
// sub-chunk products.  Blocks [0, nb_medium): one thread per medium row;
// then one block (kFloodSlots threads) per hub row.
__global__ void __launch_bounds__(kFloodSlots) k_row_beliefs(const DevGraph g, FloodPlanDev F)
{
    __shared__ XP s_x[kFloodSlots];
    if (*(volatile const int *)F.done) return;
    const int b = blockIdx.x;
    if (b < F.nb_medium) {
        const int w = b * blockDim.x + threadIdx.x;
        if (w < F.n_medium) belief_medium_item<false>(g, F, w);
        return;
    }
    belief_hub_block<false, 4>(g, F, b - F.nb_medium, s_x);
}

// ----------------------------------------------------------------------------
// Phase 2
// ----------------------------------------------------------------------------
// Typed factors of at most 32 variables: one lane per message, whole
// consecutive factors per warp (lanes_warp).  A resident grid: each warp
// takes warp records w, w + (warps in the grid), ..., keeps its largest
// residual in a register and reduces once at the end, per block into one of
// kResSlots words (per graph and per record in a batch).  One instantiation
// per combination of lanes_warp's optional parts.
template <int kFeat>
__global__ void __launch_bounds__(256, 8) k_a2v_lanes(const DevGraph g, const FloodPlanDev F, float *__restrict__ a2v,
                                                   float *__restrict__ a2v_vm, IterCtl ctl)
{
    if (*(volatile const int *)F.done) return;
    const int nw = gridDim.x * (blockDim.x >> 5);
    float dmax = 0.f;
    unsigned long long ng = 0;
    for (int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < F.n_twarps; w += nw) {  // warp-uniform
        float dd = 0.f;
        int graph = -1;
        lanes_warp<false, kFeat>(g, F, a2v, a2v_vm, w, dd, ng, graph);
        if constexpr ((kFeat & kFeatBatch) != 0) batch_residual(F, graph, dd);
        else dmax = fmaxf(dmax, dd);
    }
    if (ng) atomicAdd(ctl.guards, ng);
    if constexpr ((kFeat & kFeatBatch) != 0) return;
    const float bm = block_max(dmax);
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
    if (k < F.n_wide) wide_v2a_item<false>(g, F, a2v, k);
}

// Factors wider than a warp: one thread per edge.
__global__ void __launch_bounds__(256) k_a2v_wide(const DevGraph g, const FloodPlanDev F, float *__restrict__ a2v,
                                                  float *__restrict__ a2v_vm, IterCtl ctl)
{
    if (*(volatile const int *)F.done) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    float d = 0.f;
    unsigned long long ng = 0;
    int graph = -1;
    if (k < F.n_wide) wide_a2v_item<false>(g, F, a2v, a2v_vm, k, d, ng, graph);
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

// Phase 1 of an iteration.
void beliefs_phase(const DevGraph &g, const FloodPlanDev &P, const float *a2v_vm, cudaStream_t s)
{
    const int nb1 = (P.n_subs + P.sub_threads - 1) / P.sub_threads + P.nb_vars;
    if (nb1 > 0) k_beliefs<<<nb1, 256, 0, s>>>(g, P, a2v_vm);
    const int nb2 = P.nb_medium + P.n_hub_rows;
    if (nb2 > 0) k_row_beliefs<<<nb2, kFloodSlots, 0, s>>>(g, P);
}

// Phase 1 and phase 2 of one iteration (or one RESIDUAL level).
void flood_phases(const DevGraph &g, const FloodPlanDev &P, float *a2v, float *a2v_vm, IterCtl ctl, cudaStream_t s)
{
    beliefs_phase(g, P, a2v_vm, s);
    if (P.n_wide > 0) k_wide_v2a<<<(P.n_wide + 255) / 256, 256, 0, s>>>(g, P, a2v);
    if (P.n_twarps > 0) {
        const int feat = (P.batch.n_graphs > 0 ? kFeatBatch : 0) | (P.elevel ? kFeatLevel : 0) | (P.dres ? kFeatDres : 0);
        decltype(&k_a2v_lanes<0>) k = nullptr;
        switch (feat) {
        case 0: k = k_a2v_lanes<0>; break;
        case 1: k = k_a2v_lanes<1>; break;
        case 2: k = k_a2v_lanes<2>; break;
        case 3: k = k_a2v_lanes<3>; break;
        case 4: k = k_a2v_lanes<4>; break;
        case 5: k = k_a2v_lanes<5>; break;
        case 6: k = k_a2v_lanes<6>; break;
        default: k = k_a2v_lanes<7>; break;
        }
        // one resident grid: 8 blocks of 256 threads per SM (32 registers a thread)
        const int nb = (int)std::min<int64_t>((P.n_twarps + 7) / 8, 8 * (int64_t)num_sms());
        k<<<nb, 256, 0, s>>>(g, P, a2v, a2v_vm, ctl);
    }
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

void flood_beliefs(const DevGraph &g, const FloodPlanDev &F, const float *a2v_vm, cudaStream_t s)
{
    beliefs_phase(g, F, a2v_vm, s);
}

int flood_launches(const DevGraph &g, const FloodPlanDev &F)
{
    return (F.n_subs + F.nb_vars > 0) + (F.nb_medium + F.n_hub_rows > 0) + 2 * (F.n_wide > 0) + (F.n_twarps > 0) +
           (F.n_warps > 0) + 1;
}

}  // namespace fbp
