// Persistent level engine (sm_103a): a whole BP run of a static update
// strategy in one launch.
//
// The dependency analysis (Algorithm 2) turns the strategy into ordered
// levels; Sec. 4.3.1 executes each level in two phases (all needed
// variable-to-factor messages from the level-start state, then the level's
// factor-to-variable messages) with kernel launches per level.  Here every
// level is one step of a persistent grid, separated from the next by a
// barrier, and the convergence test runs on the device: a run of hundreds of
// levels times tens of iterations is one launch and one host synchronisation.
//
// Lane plan.  The host packs each level into warp-sized groups of lanes: one
// lane per variable of every factor the level touches, each factor whole
// inside one warp.  The lane of a factor's position j forms the incoming v->a
// message of position j (Eq. 1) by walking the variable's row; an a->v message
// updated in an earlier level of this half-iteration is read from `nxt`, any
// other from `cur` (the level-start snapshot).  The products meet in shared
// memory; then every lane whose edge belongs to the level computes its closed
// form a->v message (Eq. 4, fbp_msg.cuh).  All of a level's messages are
// computed in one pass of one lane each.
//
// Level step.  Everything a lane needs except message values (its lane
// record, its variable's row range and unary potential, the first kPre row
// entries and which buffer each comes from) is read-only, so it is fetched for
// the next level between the barrier's arrive and its wait.  After the wait a
// level costs one round of message loads, the arithmetic and the stores.
//  Cluster mode: the grid is one thread-block cluster and the barrier is the
//  hardware cluster barrier (release/acquire).  It cannot time out: all
//  blocks of a cluster are co-scheduled and run the same barrier sequence.
//  Grid mode (cooperative launch, for levels wider than a cluster): a counter
//  that only grows; one release-add per block; the block's first thread polls
//  with acquire loads, bounded by spin_limit cycles, then raises the error
//  word and every block leaves at its next barrier.
// Message buffers change between levels, so they are read and written at L2
// (ld/st.global.cg); the plan and the graph structure are read-only.
#include "fbp_flood_dev.cuh"
#include "fbp_msg.cuh"

#include <algorithm>

namespace fbp {

namespace {

constexpr int kBlock = 256;    // threads per block (grid mode)
constexpr int kClusterBlock = 512;  // threads per block in cluster mode: 16 x 16 warps hold a level
constexpr int kMaxFan = 32;    // largest factor held by one warp (larger: per-edge path)
constexpr int kPreDeep = 16;   // row entries of a lane prefetched: levels that fit the grid in one pass
constexpr int kPreWide = 8;    // levels of several passes per level (throughput, not latency, bound)
constexpr int kPreAt = 8;      // row entries per step of the per-edge path (factors wider than a warp)

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

__device__ __forceinline__ void grid_arrive(unsigned *counter)
{
    __syncthreads();
    if (threadIdx.x == 0) red_release_add(counter, 1u);
}

// Returns nonzero on timeout or when another block reported an error.
__device__ __forceinline__ int grid_wait(const unsigned *counter, unsigned target, int *err, long long spin_limit)
{
    __shared__ int s_fail;
    if (threadIdx.x == 0) {
        int fail = 0;
        const long long t0 = clock64();
        int polls = 0;
        while ((int)(ld_acquire(counter) - target) < 0) {
            if (*(volatile int *)err) { fail = 1; break; }
            if (clock64() - t0 > spin_limit) {
                atomicExch(err, 1);
                fail = 1;
                break;
            }
            if (++polls > 64) __nanosleep(20);
        }
        if (*(volatile int *)err) fail = 1;
        s_fail = fail;
    }
    __syncthreads();
    return s_fail;
}

// Dataflow execution (k_engine_df): every message a half writes starts as
// this NaN, which the encodings never produce; a reader of a message written
// at an earlier level of the half waits until the value replaces it.  The
// message is its own flag, so a relaxed load of the one word suffices.
constexpr unsigned kPending = 0x7fc0dea1u;

__device__ __forceinline__ float ld_relaxed(const float *p)
{
    float v;
    asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
    return v;
}

// v: a first load of *p.  Waits (bounded by spin_limit cycles) while the
// message is pending; on expiry raises the error word, which ends the run at
// its next grid barrier.
__device__ __forceinline__ float await_msg(const float *p, float v, const EngineArgs &A)
{
    if (__float_as_uint(v) != kPending) return v;
    const long long t0 = clock64();
    for (int n = 0;; ++n) {
        v = ld_relaxed(p);
        if (__float_as_uint(v) != kPending) return v;
        if (clock64() - t0 > A.spin_limit) {
            atomicExch(A.out + 2, 1);
            return 1.f;
        }
        if (n > 16) __nanosleep(32);
    }
}

// Incoming v->a message of edge q = (a, v) at level L without prefetch (the
// per-edge path of factors wider than a warp).
template <bool kDF>
__device__ __forceinline__ P2 v2a_at(const EngineArgs &A, const LevelPlanDev &P, int q, int L,
                                     const float *cur, const float *nxt)
{
    const int4 er = __ldg(A.erow + q);
    P2 m = dec(__ldg(A.g.phi + er.z));
    for (int k0 = er.x; k0 < er.y; k0 += kPreAt) {
        float rr[kPreAt];
#pragma unroll
        for (int u = 0; u < kPreAt; ++u) {
            rr[u] = 1.f;
            if (k0 + u < er.y) {
                const int2 ev = __ldg(P.vel + k0 + u);
                if (ev.x != q) {
                    rr[u] = ev.y < L ? __ldcg(nxt + ev.x) : __ldcg(cur + ev.x);
                    if (kDF && ev.y < L) rr[u] = await_msg(nxt + ev.x, rr[u], A);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kPreAt; ++u) {
            m = mul(m, dec(rr[u]));
            if (u & 1) resc(m);
        }
    }
    return norm_max(m);
}

// A lane's read-only state for one level.
template <int kPre>
struct Pre {
    int4 rec;          // lane record: {edge q or -1, first | n<<5 | type<<11 | target<<14, p bits, variable}
    float phi;
    int e[kPre];       // first row entries (edge ids)
    unsigned use_nxt;  // bit u: entry u was written earlier in this half-iteration
    unsigned live;     // bit u: entry u exists and is not q itself
    int kmore, kend;   // rest of the row
};

// The lane record and row range of a slot: the first of the two dependent
// rounds of a lane's read-only loads.
struct PreA {
    int4 rec;
    int2 er;
};

__device__ __forceinline__ void prefetch_a(PreA &a, const LevelPlanDev &P, int slot, int s1)
{
    a.rec = make_int4(-1, 0, 0, 0);
    a.er = make_int2(0, 0);
    if (slot >= s1) return;
    a.rec = __ldg(P.lanes + slot);
    a.er = __ldg(P.lrow + slot);  // independent of rec: both loads in flight together
}

// The second round (unary potential and the first row entries), from a
// completed first round.
template <int kPre>
__device__ __forceinline__ void prefetch_b(Pre<kPre> &s, const PreA &a, const EngineArgs &A, const LevelPlanDev &P,
                                           int La)
{
    s.rec = a.rec;
    s.use_nxt = 0u;
    s.live = 0u;
    s.kmore = s.kend = 0;
    s.phi = 1.f;
    const int2 er = a.er;
    const int q = s.rec.x;
    if (q < 0) return;
    s.phi = __ldg(A.g.phi + s.rec.w);
#pragma unroll
    for (int u = 0; u < kPre; ++u) {
        const int k = er.x + u;
        s.e[u] = 0;
        if (k < er.y) {
            const int2 ev = __ldg(P.vel + k);
            s.e[u] = ev.x;
            if (ev.x != q) s.live |= 1u << u;
            if (ev.y < La) s.use_nxt |= 1u << u;
        }
    }
    s.kmore = er.x + kPre;
    s.kend = er.y;
}

// The second round split in two for a pipeline two levels deep: the loads
// (raw row entries and phi), then, a level later, the lane state derived
// from them, so that no instruction waits on a load issued in the same level.
template <int kPre>
struct PreB {
    int2 ev[kPre];
    float phi;
};

template <int kPre>
__device__ __forceinline__ void prefetch_b_issue(PreB<kPre> &b, const PreA &a, const EngineArgs &A,
                                                 const LevelPlanDev &P)
{
    b.phi = 1.f;
#pragma unroll
    for (int u = 0; u < kPre; ++u) b.ev[u] = make_int2(-1, 0);
    if (a.rec.x < 0) return;
    b.phi = __ldg(A.g.phi + a.rec.w);
#pragma unroll
    for (int u = 0; u < kPre; ++u)
        if (a.er.x + u < a.er.y) b.ev[u] = __ldg(P.vel + a.er.x + u);
}

template <int kPre>
__device__ __forceinline__ void prefetch_b_finish(Pre<kPre> &s, const PreA &a, const PreB<kPre> &b, int La)
{
    s.rec = a.rec;
    s.phi = b.phi;
    s.use_nxt = 0u;
    s.live = 0u;
    s.kmore = a.er.x + kPre;
    s.kend = a.er.y;
    if (a.rec.x < 0) {
        s.kmore = s.kend = 0;
        return;
    }
#pragma unroll
    for (int u = 0; u < kPre; ++u) {
        s.e[u] = 0;
        if (a.er.x + u < a.er.y) {
            s.e[u] = b.ev[u].x;
            if (b.ev[u].x != a.rec.x) s.live |= 1u << u;
            if (b.ev[u].y < La) s.use_nxt |= 1u << u;
        }
    }
}

template <int kPre>
__device__ __forceinline__ void prefetch(Pre<kPre> &s, const EngineArgs &A, const LevelPlanDev &P, int La, int slot,
                                         int s1)
{
    PreA a;
    prefetch_a(a, P, slot, s1);
    prefetch_b(s, a, A, P, La);
}

// One lane's share of a level: its position's v->a product, then (if its edge
// is in the level) its factor's closed form a->v message.  Called by whole
// warps (the __syncwarp()s).
template <int kPre, bool kDF>
__device__ __forceinline__ void run_lane(const Pre<kPre> &s, const EngineArgs &A, const LevelPlanDev &P, int La,
                                         const float *cur, float *nxt, P2 *sm, float &rmax,
                                         unsigned long long &ng)
{
    const int q = s.rec.x;
    const int pk = s.rec.y;
    const bool tgt = q >= 0 && ((pk >> 14) & 1);
    const int graph = pk >> 15;
    // a graph of a batch that has stopped keeps its messages: its lanes only
    // carry them over into the next buffer
    const bool frozen = A.batch.n_graphs > 0 && q >= 0 && __ldcg(A.batch.done + graph) != 0;
    const float old = tgt ? __ldcg(cur + q) : 1.f;
    P2 m{1.f, 1.f};
    if (q >= 0 && !frozen) {
        float r[kPre];
#pragma unroll
        for (int u = 0; u < kPre; ++u)
            r[u] = ((s.live >> u) & 1u) ? (((s.use_nxt >> u) & 1u) ? __ldcg(nxt + s.e[u]) : __ldcg(cur + s.e[u]))
                                         : 1.f;
        if (kDF) {  // messages of earlier levels of this half: wait for the pending ones
#pragma unroll
            for (int u = 0; u < kPre; ++u)
                if ((s.live >> u) & (s.use_nxt >> u) & 1u) r[u] = await_msg(nxt + s.e[u], r[u], A);
        }
        m = dec(s.phi);
#pragma unroll
        for (int u = 0; u < kPre; ++u) {
            m = mul(m, dec(r[u]));
            if (u & 1) resc(m);
        }
        // the rest of a long row, kPre entries per step (entry loads first)
        for (int k0 = s.kmore; k0 < s.kend; k0 += kPre) {
            float rr[kPre];
#pragma unroll
            for (int u = 0; u < kPre; ++u) {
                rr[u] = 1.f;
                if (k0 + u < s.kend) {
                    const int2 ev = __ldg(P.vel + k0 + u);
                    if (ev.x != q) {
                        rr[u] = ev.y < La ? __ldcg(nxt + ev.x) : __ldcg(cur + ev.x);
                        if (kDF && ev.y < La) rr[u] = await_msg(nxt + ev.x, rr[u], A);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kPre; ++u) {
                m = mul(m, dec(rr[u]));
                if (u & 1) resc(m);
            }
        }
        m = norm_max(m);
    }
    const int lane = threadIdx.x & 31;
    sm[lane] = m;
    __syncwarp();
    float d = 0.f;
    if (tgt) {
        if (frozen) {
            __stcg(nxt + q, old);
        } else {
            const int first = pk & 31, n = (pk >> 5) & 63, type = (pk >> 11) & 7;
            const float p = __int_as_float(s.rec.z);
            const auto getm = [&](int j) { return sm[first + j]; };
            const P2 mu = type == kTypeTERMS ? a2v_terms(A.g, __ldg(A.g.efac + q), n, lane - first, getm)
                                             : a2v_unified(type, p, n, lane - first, getm);
            bool gd = false;
            const float r = enc_fast(mu, gd);
            ng += gd;
            d = delta_p1_fast(r, old);
            rmax = fmaxf(rmax, d);
            __stcg(nxt + q, r);
            if (A.dres) A.dres[q] = d;
        }
    }
    if (A.batch.n_graphs > 0) {
        // per-graph residual: one atomic per graph present in the warp
        const unsigned grp = __match_any_sync(0xffffffffu, q >= 0 ? graph : -1);
        const unsigned bits = __reduce_max_sync(grp, __float_as_uint(d));
        if (q >= 0 && lane == __ffs(grp) - 1 && bits) max_bits(A.batch.res + graph, bits);
    }
    __syncwarp();
}

// End of one iteration of a batch (one block): every running graph records
// its residual and iteration count and stops at its tolerance or its own
// iteration limit; the count of graphs still running is published.
__device__ __forceinline__ void batch_iteration_end(const BatchCtl &B, int it)
{
    __shared__ int s_active;
    if (threadIdx.x == 0) s_active = 0;
    __syncthreads();
    int act = 0;
    for (int gi = threadIdx.x; gi < B.n_graphs; gi += blockDim.x) {
        if (__ldcg(B.done + gi)) continue;
        const unsigned r = __ldcg(B.res + gi);
        B.res[gi] = 0u;
        B.last_res[gi] = r;
        B.iters[gi] = it;
        if (__uint_as_float(r) < __ldg(B.tol + gi)) B.done[gi] = 1;
        else if (it >= __ldg(B.max_iters + gi)) B.done[gi] = 2;
        else ++act;
    }
    act = __reduce_add_sync(0xffffffffu, act);
    if ((threadIdx.x & 31) == 0 && act) atomicAdd(&s_active, act);
    __syncthreads();
    if (threadIdx.x == 0) *B.active = s_active;
}

__device__ __forceinline__ LevelPlanDev plan_at(const EngineArgs &A, int h)
{
    return h == 0 ? A.half[0] : A.half[1];
}

template <bool kCluster, int kThreads, int kPre>
__global__ void __launch_bounds__(kThreads, 1) k_engine(EngineArgs A)
{
    __shared__ P2 s_m[kThreads];
    P2 *sm = s_m + (threadIdx.x & ~31);
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
    // A level's warp groups are dealt to warps round-robin over the blocks, so
    // that a narrow level is spread over every SM of the grid instead of
    // filling the first blocks: warp w of block b is global warp w*grid + b.
    const int lane = threadIdx.x & 31;
    const int gw = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    const int nw = nthr >> 5;
    const int my0 = gw * 32 + lane;  // this thread's slot offset in its first pass
    float *cur = A.buf[0], *nxt = A.buf[1];
    unsigned long long ng = 0;
    unsigned target = 0;
    int it, status = 1, failed = 0;
    const bool solo = gridDim.x == 1;  // one block: block barriers only
    const bool empty = A.n_halves == 0 ||
                       (A.half[0].n_levels == 0 && (A.n_halves < 2 || A.half[1].n_levels == 0));
    // Level fusion (grid mode): a level of at most A.fuse_lanes lanes and no
    // factor wider than a warp is "narrow" and runs in block 0 alone (thread
    // t takes the level's slot t); consecutive narrow levels within an
    // iteration are separated by block barriers, and the other blocks meet
    // block 0 at one grid barrier after the last of them.  Each lane computes
    // exactly what it computes in a grid-wide level.
    const bool fusing = !kCluster && !solo && A.fuse_lanes > 0;
    auto narrow = [&](const LevelPlanDev &Q, int l) {
        return fusing && __ldg(Q.lane_ptr + l + 1) - __ldg(Q.lane_ptr + l) <= A.fuse_lanes &&
               __ldg(Q.big_ptr + l + 1) == __ldg(Q.big_ptr + l);
    };
    auto first_slot = [&](bool nar, int s0, int s1) {
        return nar ? (blockIdx.x == 0 ? s0 + (int)threadIdx.x : s1) : s0 + my0;
    };
    Pre<kPre> pre;
    bool nar = false;
    if (!empty) {
        int h0 = 0;
        while (plan_at(A, h0).n_levels == 0) ++h0;
        const LevelPlanDev P0 = plan_at(A, h0);
        nar = narrow(P0, 0);
        const int s0 = __ldg(P0.lane_ptr), s1 = __ldg(P0.lane_ptr + 1);
        prefetch(pre, A, P0, P0.level_base, first_slot(nar, s0, s1), s1);
    }
    for (it = 1; it <= A.max_iters && !failed && !empty; ++it) {
        float rmax = 0.f;
        for (int h = 0; h < A.n_halves && !failed; ++h) {
            const LevelPlanDev P = plan_at(A, h);
            for (int L = 0; L < P.n_levels; ++L) {
                const int La = L + P.level_base;
                const int s0 = __ldg(P.lane_ptr + L), s1 = __ldg(P.lane_ptr + L + 1);
                // the next level (next half, or the next iteration's first
                // level): its lane records are requested before this level's
                // work and its dependent loads between the barrier's arrive and
                // wait, so that neither round trip adds to the level's time
                int Ln = L + 1, hn = h;
                LevelPlanDev Pn = P;
                while (Ln >= Pn.n_levels) {
                    Ln = 0;
                    hn = hn + 1 < A.n_halves ? hn + 1 : 0;
                    Pn = plan_at(A, hn);
                    if (Pn.n_levels > 0) break;
                }
                const bool last_of_iteration = L + 1 == P.n_levels && h + 1 == A.n_halves;
                const bool nar_n = narrow(Pn, Ln);
                // a narrow level followed by a narrow one of the same
                // iteration: block 0 alone, no grid barrier in between
                const bool fused = nar && nar_n && !last_of_iteration;
                PreA next;
                {
                    const int n0 = __ldg(Pn.lane_ptr + Ln), n1 = __ldg(Pn.lane_ptr + Ln + 1);
                    prefetch_a(next, Pn, first_slot(nar_n, n0, n1), n1);
                }
                run_lane<kPre, false>(pre, A, P, La, cur, nxt, sm, rmax, ng);
                for (int slot = nar ? s1 : s0 + my0 + nthr; slot < s1; slot += nthr) {  // levels wider than the grid
                    Pre<kPre> more;
                    prefetch(more, A, P, La, slot, s1);
                    run_lane<kPre, false>(more, A, P, La, cur, nxt, sm, rmax, ng);
                }
                // factors wider than a warp: one thread per edge
                const int b0 = __ldg(P.big_ptr + L), b1 = __ldg(P.big_ptr + L + 1);
                for (int b = b0 + tid; b < b1; b += nthr) {
                    const int e = __ldg(P.big + b);
                    const int a = __ldg(A.g.efac + e);
                    const int lo = __ldg(A.g.fptr + a), n = __ldg(A.g.fptr + a + 1) - lo;
                    const P2 mu = a2v_unified(__ldg(A.g.ftype + a), __ldg(A.g.fparam + a), n, e - lo,
                                              [&](int j) { return v2a_at<false>(A, P, lo + j, La, cur, nxt); });
                    bool gd = false;
                    const float r = enc_fast(mu, gd);
                    ng += gd;
                    const float d = delta_p1_fast(r, __ldcg(cur + e));
                    rmax = fmaxf(rmax, d);
                    __stcg(nxt + e, r);
                    if (A.dres) A.dres[e] = d;
                }
                if (L + 1 == P.n_levels && h + 1 == A.n_halves) {
                    const float bm = block_max(rmax);
                    if (threadIdx.x == 0 && bm > 0.f) max_bits(A.res + (it - 1), __float_as_uint(bm));
                }
                // A one-block grid (or block 0 inside a run of fused narrow
                // levels) needs no grid barrier: __syncthreads orders the
                // block's message stores before the next level's loads.
                if (kCluster) {
                    cluster_arrive();
                } else if (!solo && !fused) {
                    grid_arrive(A.bar);
                    target += gridDim.x;
                }
                // the dependent round uses its loads at once: inside the barrier
                prefetch_b(pre, next, A, Pn, Ln + Pn.level_base);
                nar = nar_n;
                if (kCluster) {
                    cluster_wait();
                } else if (solo || fused) {
                    if (blockIdx.x == 0) __syncthreads();
                } else if (grid_wait(A.bar, target, A.out + 2, A.spin_limit)) {
                    failed = 1;
                    break;
                }
            }
            float *t = cur;
            cur = nxt;
            nxt = t;
        }
        if (failed) break;
        if (A.batch.n_graphs > 0) {
            if (blockIdx.x == 0) batch_iteration_end(A.batch, it);
            if (kCluster) {
                cluster_arrive();
                cluster_wait();
            } else if (solo) {
                __syncthreads();
            } else {
                grid_arrive(A.bar);
                target += gridDim.x;
                if (grid_wait(A.bar, target, A.out + 2, A.spin_limit)) {
                    failed = 1;
                    break;
                }
            }
            if (*(volatile int *)A.batch.active == 0) {
                status = 0;
                break;
            }
            continue;
        }
        const float r = __uint_as_float(*(volatile unsigned *)(A.res + (it - 1)));
        if (r < A.tol) {
            status = 0;
            break;
        }
    }
    if (empty) {
        status = 0;
        it = 1;
    }
    if (ng) atomicAdd(A.guards, ng);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.out[0] = it > A.max_iters ? A.max_iters : it;
        A.out[1] = failed ? -1 : status;
    }
}

// The dataflow engine: the same levels and the same arithmetic as k_engine,
// without a grid barrier between levels.  At the start of a half every
// message the half writes is set pending (then one grid barrier); a lane
// waits only for the messages it reads that earlier levels of the half write
// (await_msg), and reads every other message from the level-start buffer,
// which nothing writes during the half.  So every lane reads exactly the
// values the level-by-level execution gives it, and a level starts as soon as
// its own inputs exist instead of when the slowest lane of the previous level
// finishes.  A half ends with a grid barrier (all reads of the old buffer
// done) before the buffers swap.  No wait can deadlock: a lane waits only on
// lanes of lower levels of the same half, every thread takes its levels in
// order, and the cooperative launch keeps every block resident.  Every wait
// is bounded (spin_limit).  Static strategies only (every edge is written
// once per half).
template <int kPre>
__global__ void __launch_bounds__(kBlock, 1) k_engine_df(EngineArgs A)
{
    __shared__ P2 s_m[kBlock];
    P2 *sm = s_m + (threadIdx.x & ~31);
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const int gw = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    const int my0 = gw * 32 + lane;
    float *cur = A.buf[0], *nxt = A.buf[1];
    unsigned long long ng = 0;
    unsigned target = 0;
    int it, status = 1, failed = 0;
    const bool empty = A.n_halves == 0 ||
                       (A.half[0].n_levels == 0 && (A.n_halves < 2 || A.half[1].n_levels == 0));
    Pre<kPre> pre;
    for (it = 1; it <= A.max_iters && !failed && !empty; ++it) {
        float rmax = 0.f;
        for (int h = 0; h < A.n_halves && !failed; ++h) {
            const LevelPlanDev P = plan_at(A, h);
            for (int e = tid; e < A.g.ne; e += nthr) __stcg(nxt + e, __uint_as_float(kPending));
            // plan pipeline: level L's lane state, level L+1's loads, level L+2's records
            PreA rec1;
            PreB<kPre> raw1;
            if (P.n_levels > 0)
                prefetch(pre, A, P, P.level_base, __ldg(P.lane_ptr) + my0, __ldg(P.lane_ptr + 1));
            if (P.n_levels > 1) {
                prefetch_a(rec1, P, __ldg(P.lane_ptr + 1) + my0, __ldg(P.lane_ptr + 2));
                prefetch_b_issue(raw1, rec1, A, P);
            }
            grid_arrive(A.bar);
            target += gridDim.x;
            if (grid_wait(A.bar, target, A.out + 2, A.spin_limit)) {
                failed = 1;
                break;
            }
            for (int L = 0; L < P.n_levels; ++L) {
                const int La = L + P.level_base;
                const int s0 = __ldg(P.lane_ptr + L), s1 = __ldg(P.lane_ptr + L + 1);
                PreA rec2;
                if (L + 2 < P.n_levels) prefetch_a(rec2, P, __ldg(P.lane_ptr + L + 2) + my0, __ldg(P.lane_ptr + L + 3));
                run_lane<kPre, true>(pre, A, P, La, cur, nxt, sm, rmax, ng);
                for (int slot = s0 + my0 + nthr; slot < s1; slot += nthr) {  // levels wider than the grid
                    Pre<kPre> more;
                    prefetch(more, A, P, La, slot, s1);
                    run_lane<kPre, true>(more, A, P, La, cur, nxt, sm, rmax, ng);
                }
                const int b0 = __ldg(P.big_ptr + L), b1 = __ldg(P.big_ptr + L + 1);
                for (int b = b0 + tid; b < b1; b += nthr) {  // factors wider than a warp
                    const int e = __ldg(P.big + b);
                    const int a = __ldg(A.g.efac + e);
                    const int lo = __ldg(A.g.fptr + a), n = __ldg(A.g.fptr + a + 1) - lo;
                    const P2 mu = a2v_unified(__ldg(A.g.ftype + a), __ldg(A.g.fparam + a), n, e - lo,
                                              [&](int j) { return v2a_at<true>(A, P, lo + j, La, cur, nxt); });
                    bool gd = false;
                    const float r = enc_fast(mu, gd);
                    ng += gd;
                    rmax = fmaxf(rmax, delta_p1_fast(r, __ldcg(cur + e)));
                    __stcg(nxt + e, r);
                }
                if (L + 1 < P.n_levels) prefetch_b_finish(pre, rec1, raw1, La + 1);
                if (L + 2 < P.n_levels) {
                    prefetch_b_issue(raw1, rec2, A, P);
                    rec1 = rec2;
                }
            }
            if (h + 1 == A.n_halves) {
                const float bm = block_max(rmax);
                if (threadIdx.x == 0 && bm > 0.f) max_bits(A.res + (it - 1), __float_as_uint(bm));
            }
            grid_arrive(A.bar);
            target += gridDim.x;
            if (grid_wait(A.bar, target, A.out + 2, A.spin_limit)) {
                failed = 1;
                break;
            }
            float *t = cur;
            cur = nxt;
            nxt = t;
        }
        if (failed) break;
        if (A.batch.n_graphs > 0) {
            if (blockIdx.x == 0) batch_iteration_end(A.batch, it);
            grid_arrive(A.bar);
            target += gridDim.x;
            if (grid_wait(A.bar, target, A.out + 2, A.spin_limit)) {
                failed = 1;
                break;
            }
            if (*(volatile int *)A.batch.active == 0) {
                status = 0;
                break;
            }
            continue;
        }
        const float r = __uint_as_float(*(volatile unsigned *)(A.res + (it - 1)));
        if (r < A.tol) {
            status = 0;
            break;
        }
    }
    if (empty) {
        status = 0;
        it = 1;
    }
    if (ng) atomicAdd(A.guards, ng);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.out[0] = it > A.max_iters ? A.max_iters : it;
        A.out[1] = failed ? -1 : status;
    }
}

// ---------------------------------------------------------------------------
// Batch queue: a whole batch in one launch.  Thread-block clusters of
// kCl (8 or 16) blocks take members from a queue (largest first) and run
// each to its own stopping rule: a flooding member by the flooding items of
// fbp_flood_dev.cuh over its own ranges of the union's flooding plan, a
// static member by the level engine's lanes over its own level lists.  The
// blocks of a cluster are co-scheduled by the hardware, so a barrier among
// them cannot wait on a block that is not running; clusters never wait on
// one another, so the launch needs no co-residency beyond a cluster.  The
// barrier is the grid barrier's counter scheme on the cluster's own word,
// every wait bounded by spin_limit (an expiry sets the error word, which
// every cluster sees at its next barrier).  Data the cluster's blocks write
// for one another between phases is read with coherent loads.
// ---------------------------------------------------------------------------
constexpr int kQueueBlock = 256;
constexpr int kQueuePre = 4;  // row entries per prefetch step (even: same rescaling points as the engine)

__device__ __forceinline__ unsigned cluster_ctarank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned cluster_id_x()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}

template <int kCl>
struct ClusterBar {
    unsigned *ctr;
    unsigned target;
    int *err;
    long long spin;
    __device__ __forceinline__ int sync()
    {
        grid_arrive(ctr);
        target += kCl;
        return grid_wait(ctr, target, err, spin);
    }
};

template <int kCl>
__global__ void __launch_bounds__(kQueueBlock, 3) k_batch_queue(const QueueArgs Q)
{
    static_assert(kQueueBlock == kFloodSlots, "a block combines one hub row");
    __shared__ P2 s_m[kQueueBlock];
    __shared__ XP s_x[kFloodSlots];
    P2 *sm = s_m + (threadIdx.x & ~31);
    const int r = (int)cluster_ctarank(), c = (int)cluster_id_x();
    const int gt = r * kQueueBlock + (int)threadIdx.x, nt = kCl * kQueueBlock;  // thread in the cluster
    const int gw = gt >> 5, nwp = nt >> 5;                                              // warp in the cluster
    EngineArgs A;
    A.g = Q.g;
    A.erow = Q.erow;
    ClusterBar<kCl> bar{Q.cbar + c, 0u, Q.err, Q.spin_limit};
    int32_t *word = Q.cword + 4 * c;
    unsigned long long ng = 0;
    bool failed = false;
    for (;;) {
        if (r == 0 && threadIdx.x == 0) word[0] = atomicAdd(Q.queue, 1);
        if (bar.sync()) break;
        const int pos = __ldcg(word);
        if (pos >= Q.n_members) break;
        const int m = __ldg(Q.order + pos);
        const MemberDev &M = Q.members[m];
        int it, status = 1;
        unsigned rbits = 0;
        float *cur = Q.a2v, *nxt = Q.a2v_alt;
        const int kind = M.kind, max_iters = M.max_iters;
        const float tol = M.tol;
        const bool empty_static = kind > 0 && M.half[0].n_levels == 0 && (kind < 2 || M.half[1].n_levels == 0);
        if (empty_static) {  // as the engine: nothing to update, converged at once
            it = 1;
            status = 0;
        }
        for (it = 1; !empty_static && it <= max_iters; ++it) {
            float rmax = 0.f;
            if (kind == 0) {
                // the sub-chunk products and the short rows' beliefs share no data
                for (int k = M.sub0 + gt; k < M.sub1; k += nt) fdev::sub_product_item<true>(Q.g, Q.F, Q.a2v_vm, k);
                for (int v = M.v0 + gt; v < M.v1; v += nt) fdev::belief_var_item<true>(Q.g, Q.F, Q.a2v_vm, v);
                if ((failed = bar.sync())) break;
                for (int w = M.med0 + gt; w < M.med1; w += nt) fdev::belief_medium_item<true>(Q.g, Q.F, w);
                for (int hr = M.hub0 + r; hr < M.hub1; hr += kCl) fdev::belief_hub_block<true, 1>(Q.g, Q.F, hr, s_x);
                if ((failed = bar.sync())) break;
                if (M.wide1 > M.wide0) {
                    for (int k = M.wide0 + gt; k < M.wide1; k += nt) fdev::wide_v2a_item<true>(Q.g, Q.F, Q.a2v, k);
                    if ((failed = bar.sync())) break;
                }
                for (int w = M.tw0 + gw; w < M.tw1; w += nwp) {
                    float dd = 0.f;
                    int graph = -1;
                    fdev::lanes_warp<true, 0>(Q.g, Q.F, Q.a2v, Q.a2v_vm, w, dd, ng, graph);
                    rmax = fmaxf(rmax, dd);
                }
                for (int k = M.wide0 + gt; k < M.wide1; k += nt) {
                    float dd = 0.f;
                    int graph = -1;
                    fdev::wide_a2v_item<true>(Q.g, Q.F, Q.a2v, Q.a2v_vm, k, dd, ng, graph);
                    rmax = fmaxf(rmax, dd);
                }
            } else {
                for (int h = 0; h < kind && !failed; ++h) {
                    const LevelPlanDev P = Q.members[m].half[h];  // from memory: no local copy indexed at run time
                    for (int L = 0; L < P.n_levels; ++L) {
                        const int La = L + P.level_base;
                        const int s0 = __ldg(P.lane_ptr + L), s1 = __ldg(P.lane_ptr + L + 1);
                        // slots come in whole warps (lane_ptr and the stride are multiples of 32)
                        for (int slot = s0 + gt; slot < s1; slot += nt) {
                            Pre<kQueuePre> pre;
                            prefetch(pre, A, P, La, slot, s1);
                            run_lane<kQueuePre, false>(pre, A, P, La, cur, nxt, sm, rmax, ng);
                        }
                        // factors wider than a warp: one thread per edge
                        const int b0 = __ldg(P.big_ptr + L), b1 = __ldg(P.big_ptr + L + 1);
                        for (int b = b0 + gt; b < b1; b += nt) {
                            const int e = __ldg(P.big + b);
                            const int a = __ldg(A.g.efac + e);
                            const int lo = __ldg(A.g.fptr + a), n = __ldg(A.g.fptr + a + 1) - lo;
                            const P2 mu = a2v_unified(__ldg(A.g.ftype + a), __ldg(A.g.fparam + a), n, e - lo,
                                                      [&](int j) { return v2a_at<false>(A, P, lo + j, La, cur, nxt); });
                            bool gd = false;
                            const float rr = enc_fast(mu, gd);
                            ng += gd;
                            rmax = fmaxf(rmax, delta_p1_fast(rr, __ldcg(cur + e)));
                            __stcg(nxt + e, rr);
                        }
                        if ((failed = bar.sync())) break;
                    }
                    float *t = cur;
                    cur = nxt;
                    nxt = t;
                }
                if (failed) break;
            }
            // the iteration's residual: warp max, one atomic per warp, read
            // and cleared by block 0 of the cluster, which decides the stop
            const unsigned bits = __reduce_max_sync(0xffffffffu, __float_as_uint(rmax));
            if ((threadIdx.x & 31) == 0 && bits) max_bits(Q.cres + c, bits);
            if ((failed = bar.sync())) break;
            if (r == 0 && threadIdx.x == 0) {
                const unsigned rb = atomicExch(Q.cres + c, 0u);
                word[1] = __uint_as_float(rb) < tol ? 1 : it >= max_iters ? 2 : 0;
                word[2] = (int)rb;
            }
            if ((failed = bar.sync())) break;
            const int stop = __ldcg(word + 1);
            rbits = (unsigned)__ldcg(word + 2);
            if (stop) {
                status = stop == 1 ? 0 : 1;
                break;
            }
        }
        if (failed) break;
        if (!empty_static && it > max_iters) it = max_iters;
        // a static member ends with its messages in the first buffer
        if (kind > 0 && cur != Q.a2v)
            for (int e = M.e0 + gt; e < M.e1; e += nt) __stcg(Q.a2v + e, __ldcg(cur + e));
        if (r == 0 && threadIdx.x == 0) {
            Q.out_iters[m] = it;
            Q.out_status[m] = status;
            Q.out_res[m] = rbits;
        }
    }
    if (ng) atomicAdd(Q.guards, ng);
}

}  // namespace

int engine_block() { return kBlock; }
int engine_max_fan() { return kMaxFan; }

// Blocks of a cooperative grid that can be co-resident: for the shallow
// (wide-level) variant, and for the deep-prefetch variant (more registers).
static int cap_of(const void *kernel)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0);
    return per_sm * num_sms() > 0 ? per_sm * num_sms() : 1;
}

int engine_max_grid()
{
    static int cap = 0;
    if (!cap) cap = std::min(cap_of((const void *)k_engine<false, kBlock, kPreWide>),
                             cap_of((const void *)k_engine_df<kPreWide>));
    return cap;
}

static int engine_deep_grid()
{
    static int cap = 0;
    if (!cap) cap = std::min(cap_of((const void *)k_engine<false, kBlock, kPreDeep>),
                             cap_of((const void *)k_engine_df<kPreDeep>));
    return cap;
}

// Largest cluster (16 or 8 blocks, 0 if none) that can be scheduled for the
// engine's block shape on this device.
int engine_cluster_size()
{
    static int size = -1;
    if (size < 0) {
        size = 0;
        cudaFuncSetAttribute(k_engine<true, kClusterBlock, kPreDeep>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        for (int c : {16, 8}) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(c);
            cfg.blockDim = dim3(kClusterBlock);
            cudaLaunchAttribute attr;
            attr.id = cudaLaunchAttributeClusterDimension;
            attr.val.clusterDim.x = c;
            attr.val.clusterDim.y = 1;
            attr.val.clusterDim.z = 1;
            cfg.attrs = &attr;
            cfg.numAttrs = 1;
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, k_engine<true, kClusterBlock, kPreDeep>, &cfg) == cudaSuccess && n > 0) {
                size = c;
                break;
            }
            cudaGetLastError();
        }
    }
    return size;
}

cudaError_t launch_engine(const EngineArgs &a, int grid, int cluster, cudaStream_t s)
{
    EngineArgs args = a;
    if (cluster > 0) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cluster);
        cfg.blockDim = dim3(kClusterBlock);
        cfg.stream = s;
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = cluster;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, k_engine<true, kClusterBlock, kPreDeep>, args);
    }
    const int cap = engine_max_grid();
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    void *params[] = {&args};
    // levels that the grid holds in one pass are latency bound: prefetch
    // deep (when the grid fits that variant's co-residency); wider levels run
    // several passes and are throughput bound: the lighter variant, whose
    // grid may hold two blocks per SM.  Both compute the same messages.
    const bool deep = grid <= engine_deep_grid() && (long long)a.max_lanes <= (long long)grid * kBlock;
    const void *kernel = a.dataflow ? (deep ? (const void *)k_engine_df<kPreDeep> : (const void *)k_engine_df<kPreWide>)
                                    : (deep ? (const void *)k_engine<false, kBlock, kPreDeep>
                                            : (const void *)k_engine<false, kBlock, kPreWide>);
    return cudaLaunchCooperativeKernel(kernel, dim3(grid), dim3(kBlock), params, 0, s);
}

namespace {

const void *queue_kernel(int cluster)
{
    return cluster == 16 ? (const void *)k_batch_queue<16> : (const void *)k_batch_queue<8>;
}

cudaLaunchConfig_t queue_config(int cluster, int clusters, cudaStream_t s, cudaLaunchAttribute *attr)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster * clusters);
    cfg.blockDim = dim3(kQueueBlock);
    cfg.stream = s;
    attr->id = cudaLaunchAttributeClusterDimension;
    attr->val.clusterDim.x = cluster;
    attr->val.clusterDim.y = 1;
    attr->val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

}  // namespace

int batch_queue_clusters(int cluster)
{
    static int clusters[2] = {-1, -1};
    if (cluster != 8 && cluster != 16) return 0;
    int &n = clusters[cluster == 16];
    if (n >= 0) return n;
    n = 0;
    if (cluster == 16 &&
        cudaFuncSetAttribute(queue_kernel(16), cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return n;
    }
    cudaLaunchAttribute attr;
    const cudaLaunchConfig_t cfg = queue_config(cluster, 64, nullptr, &attr);
    if (cudaOccupancyMaxActiveClusters(&n, queue_kernel(cluster), &cfg) != cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    return n;
}

cudaError_t launch_batch_queue(const QueueArgs &q, int cluster, int clusters, cudaStream_t s)
{
    if (clusters < 1 || (cluster != 8 && cluster != 16)) return cudaErrorInvalidConfiguration;
    QueueArgs args = q;
    cudaLaunchAttribute attr;
    const cudaLaunchConfig_t cfg = queue_config(cluster, clusters, s, &attr);
    return cluster == 16 ? cudaLaunchKernelEx(&cfg, k_batch_queue<16>, args)
                         : cudaLaunchKernelEx(&cfg, k_batch_queue<8>, args);
}

}  // namespace fbp
