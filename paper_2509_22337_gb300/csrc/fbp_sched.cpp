// Graph layout and dependency analysis on the host.
#include "fbp_sched.h"

#include <algorithm>
#include <memory>
#include <cstring>
#include <limits>
#include <numeric>
#include <thread>

namespace fbp {

void build_host_csr(int32_t nv, int32_t na, const int64_t *fptr, const int32_t *fvars,
                    const uint8_t *ftype, const float *fparam, HostCSR &h)
{
    h.nv = nv;
    h.na = na;
    h.ne = (int32_t)fptr[na];
    const int64_t ne = h.ne;
    const int threads = host_threads_all();
    h.fptr.assign(fptr, fptr + na + 1);
    h.ftype.assign(ftype, ftype + na);
    h.fparam.assign(fparam, fparam + na);
    h.fvars.resize(ne);
    h.efac.resize(ne);
    parallel_for(na, threads, 1 << 14, [&](int64_t b, int64_t e) {
        for (int64_t a = b; a < e; ++a)
            for (int64_t k = fptr[a]; k < fptr[a + 1]; ++k) {
                h.fvars[k] = fvars[k];
                h.efac[k] = (int32_t)a;
            }
    });
    // The transpose, a stable counting sort of the edges by variable over P
    // contiguous parts of the edge range: each part counts its variables; a
    // variable's row takes part 0's edges, then part 1's, ...; each part
    // scatters its edges in order, so every row lists its edges in
    // ascending id, as the one-part (serial) sort does.  The parts' counters
    // take P * nv words, so P is bounded by a budget of 2^26 words.
    const int64_t parts = std::max<int64_t>(
        1, std::min<int64_t>({(int64_t)threads, ne / 65536, (int64_t(1) << 26) / std::max<int64_t>(nv, 1)}));
    const int64_t step = (ne + parts - 1) / parts;
    std::vector<std::unique_ptr<int32_t[]>> cnt(parts);
    for (auto &c : cnt) c.reset(new int32_t[std::max<int64_t>(nv, 1)]);
    parallel_for(parts, (int)parts, 1, [&](int64_t pb, int64_t pe) {
        for (int64_t k = pb; k < pe; ++k) {
            int32_t *c = cnt[k].get();
            std::fill(c, c + nv, 0);
            for (int64_t e = k * step, end = std::min(ne, (k + 1) * step); e < end; ++e) c[fvars[e]]++;
        }
    });
    h.vptr.assign((size_t)nv + 1, 0);
    parallel_for(nv, threads, 1 << 16, [&](int64_t b, int64_t e) {
        for (int64_t v = b; v < e; ++v) {
            int32_t sum = 0;
            for (int64_t k = 0; k < parts; ++k) {
                const int32_t c = cnt[k][v];
                cnt[k][v] = sum;  // part k's first slot within the row
                sum += c;
            }
            h.vptr[v + 1] = sum;
        }
    });
    for (int32_t v = 0; v < nv; ++v) h.vptr[v + 1] += h.vptr[v];
    h.vedge.resize(ne);
    parallel_for(parts, (int)parts, 1, [&](int64_t pb, int64_t pe) {
        for (int64_t k = pb; k < pe; ++k) {
            int32_t *c = cnt[k].get();
            for (int64_t e = k * step, end = std::min(ne, (k + 1) * step); e < end; ++e) {
                const int32_t v = fvars[e];
                h.vedge[h.vptr[v] + c[v]++] = (int32_t)e;
            }
        }
    });
}

// TOPO: depth of every variable over the "premise -> output" relation of the
// factors (a variable without a defining factor has depth 0; a factor with no
// premises defines depth 0).  Returns false on a cycle.
static bool variable_depths(const HostCSR &h, std::vector<int64_t> &depth)
{
    std::vector<int32_t> pending(h.nv, 0);     // premises of defining factors still unresolved
    std::vector<int32_t> uptr(h.nv + 1, 0);     // factors in which a variable is a premise
    for (int32_t a = 0; a < h.na; ++a) {
        const int64_t lo = h.fptr[a], hi = h.fptr[a + 1];
        if (hi <= lo) continue;
        pending[h.fvars[hi - 1]] += (int32_t)(hi - 1 - lo);
        for (int64_t e = lo; e < hi - 1; ++e) uptr[h.fvars[e] + 1]++;
    }
    for (int32_t v = 0; v < h.nv; ++v) uptr[v + 1] += uptr[v];
    std::vector<int32_t> uses(uptr[h.nv]);
    std::vector<int32_t> pos(uptr.begin(), uptr.end() - 1);
    for (int32_t a = 0; a < h.na; ++a)
        for (int64_t e = h.fptr[a]; e + 1 < h.fptr[a + 1]; ++e) uses[pos[h.fvars[e]]++] = a;
    depth.assign(h.nv, 0);
    std::vector<int32_t> ready;
    ready.reserve(h.nv);
    for (int32_t v = 0; v < h.nv; ++v)
        if (pending[v] == 0) ready.push_back(v);
    for (size_t r = 0; r < ready.size(); ++r) {
        const int32_t u = ready[r];
        for (int32_t k = uptr[u]; k < uptr[u + 1]; ++k) {
            const int32_t a = uses[k];
            const int32_t y = h.fvars[h.fptr[a + 1] - 1];
            depth[y] = std::max(depth[y], depth[u] + 1);
            if (--pending[y] == 0) ready.push_back(y);
        }
    }
    return (int32_t)ready.size() == h.nv;
}

void backward_ranks(const std::vector<int64_t> &fwd, std::vector<int64_t> &bwd)
{
    int64_t mx = 0;
    for (int64_t r : fwd) mx = std::max(mx, r);
    bwd.resize(fwd.size());
    for (size_t e = 0; e < fwd.size(); ++e) bwd[e] = mx - fwd[e];
}

int build_ranks(const HostCSR &h, const fbp_schedule_spec &spec, int half, std::vector<int64_t> &rank)
{
    rank.assign(h.ne, 0);
    switch (spec.strategy) {
    case FBP_PARALL:
        return FBP_OK;
    case FBP_SEQFIX:
        for (int32_t e = 0; e < h.ne; ++e) rank[e] = spec.edge_rank ? spec.edge_rank[e] : e;
        return FBP_OK;
    case FBP_CUSTOM_RANK:
        if (!spec.edge_rank) return fail(FBP_ERR_INVALID_ARG, "CUSTOM_RANK needs edge_rank");
        for (int32_t e = 0; e < h.ne; ++e) rank[e] = spec.edge_rank[e];
        return FBP_OK;
    case FBP_TOPO:
    case FBP_TOPO_FB: {
        if (spec.factor_rank) {
            for (int32_t e = 0; e < h.ne; ++e) rank[e] = spec.factor_rank[h.efac[e]];
        } else {
            std::vector<int64_t> depth;
            if (!variable_depths(h, depth))
                return fail(FBP_ERR_SCHEDULE, "TOPO: the premise->output relation has a cycle");
            for (int32_t a = 0; a < h.na; ++a) {
                const int64_t lo = h.fptr[a], hi = h.fptr[a + 1];
                for (int64_t e = lo; e < hi; ++e) rank[e] = depth[h.fvars[hi - 1]];
            }
        }
        if (half == 1) {
            std::vector<int64_t> fwd = std::move(rank);
            backward_ranks(fwd, rank);
        }
        return FBP_OK;
    }
    default:
        return fail(FBP_ERR_INVALID_ARG, "unknown strategy %d", spec.strategy);
    }
}

// Canonical order (Definition 2): edges by (rank, edge id).  `edges` (NULL =
// all edges) lists edge ids in ascending order.  Ranks spanning a range no
// wider than a few times the edge count (every strategy's but a sparse
// custom one) are placed by a stable counting sort, which keeps the ascending
// id order inside each rank; others by a comparison sort of (rank, id) pairs.
static void canonical_order(const int64_t *rank, const int32_t *edges, int64_t n, std::vector<int32_t> &le)
{
    le.resize(n);
    if (n == 0) return;
    auto id = [edges](int64_t i) { return edges ? edges[i] : (int32_t)i; };
    int64_t lo = rank[id(0)], hi = lo;
    for (int64_t i = 1; i < n; ++i) {
        const int64_t r = rank[id(i)];
        lo = std::min(lo, r);
        hi = std::max(hi, r);
    }
    const uint64_t span = (uint64_t)hi - (uint64_t)lo;  // exact for hi >= lo
    if (span <= (uint64_t)(4 * n + 1024)) {
        std::vector<int64_t> start(span + 2, 0);
        for (int64_t i = 0; i < n; ++i) ++start[(uint64_t)rank[id(i)] - (uint64_t)lo + 1];
        for (uint64_t k = 1; k < span + 2; ++k) start[k] += start[k - 1];
        for (int64_t i = 0; i < n; ++i) {
            const int32_t e = id(i);
            le[start[(uint64_t)rank[e] - (uint64_t)lo]++] = e;
        }
        return;
    }
    struct Key {
        int64_t r;
        int32_t e;
    };
    std::vector<Key> keys(n);
    for (int64_t i = 0; i < n; ++i) keys[i] = Key{rank[id(i)], id(i)};
    std::sort(keys.begin(), keys.end(), [](const Key &x, const Key &y) { return x.r != y.r ? x.r < y.r : x.e < y.e; });
    for (int64_t i = 0; i < n; ++i) le[i] = keys[i].e;
}

// Algorithm 2 (Sec. 4.2.3) without the sequential scan over NextSet.  NextSet
// is always a contiguous run [s, i) of the canonical order, and e_i = (a, v)
// ends it exactly when N_E(e_i) (Definition 1) holds an edge of lower rank at a
// position >= s.  Lower rank means a position before the first edge of e_i's
// rank class, so with
//   dep(i) = the largest position p < classStart(i) of an edge (a*, v*) with
//            v* in N(a) \ v and a* != a
// (one binary search per variable v* in its positions, sorted) the cut test
// is dep(i) >= s.  dep is independent per edge and runs on several threads;
// the cuts follow in one pass.  With a single class nothing can cut, and the
// edges form one level.
void dependency_levels(const HostCSR &h, const int64_t *rank, const int32_t *edges, int64_t n,
                       std::vector<int64_t> &lp, std::vector<int32_t> &le)
{
    canonical_order(rank, edges, n, le);
    lp.assign(1, 0);
    if (n == 0) return;
    if (rank[le[0]] == rank[le[n - 1]]) {
        lp.push_back(n);
        return;
    }
    const int T = host_threads();
    // position of every scheduled edge; -1 for the others
    std::vector<int32_t> pos(h.ne, -1);
    parallel_for(n, T, 1 << 16, [&](int64_t b, int64_t e) {
        for (int64_t i = b; i < e; ++i) pos[le[i]] = (int32_t)i;
    });
    // first position of each position's rank class
    std::vector<int32_t> cstart(n);
    cstart[0] = 0;
    for (int64_t i = 1; i < n; ++i) cstart[i] = rank[le[i]] == rank[le[i - 1]] ? cstart[i - 1] : (int32_t)i;
    // every variable's scheduled edges as ascending positions
    std::vector<int32_t> vp(h.nv + 1, 0), vpos(n);
    if (!edges) {
        std::copy(h.vptr.begin(), h.vptr.end(), vp.begin());
    } else {
        parallel_for(h.nv, T, 1 << 14, [&](int64_t b, int64_t e) {
            for (int64_t v = b; v < e; ++v) {
                int32_t c = 0;
                for (int32_t k = h.vptr[v]; k < h.vptr[v + 1]; ++k) c += pos[h.vedge[k]] >= 0;
                vp[v + 1] = c;
            }
        });
        for (int32_t v = 0; v < h.nv; ++v) vp[v + 1] += vp[v];
    }
    parallel_for(h.nv, T, 1 << 14, [&](int64_t b, int64_t e) {
        for (int64_t v = b; v < e; ++v) {
            int32_t *out = vpos.data() + vp[v], k = 0;
            for (int32_t r = h.vptr[v]; r < h.vptr[v + 1]; ++r)
                if (pos[h.vedge[r]] >= 0) out[k++] = pos[h.vedge[r]];
            std::sort(out, out + k);
        }
    });
    std::vector<int32_t> dep(n);
    parallel_for(n, T, 1 << 14, [&](int64_t b, int64_t e) {
        for (int64_t i = b; i < e; ++i) {
            const int32_t ei = le[i], a = h.efac[ei], v = h.fvars[ei], cs = cstart[i];
            int32_t best = -1;
            for (int64_t q = h.fptr[a]; q < h.fptr[a + 1]; ++q) {
                const int32_t vs = h.fvars[q];
                if (vs == v) continue;
                const int32_t *b0 = vpos.data() + vp[vs], *b1 = vpos.data() + vp[vs + 1];
                const int32_t *it = std::lower_bound(b0, b1, cs);
                if (it != b0 && it[-1] == pos[q]) --it;  // a's own edge into vs does not count
                if (it != b0) best = std::max(best, it[-1]);
            }
            dep[i] = best;
        }
    });
    int64_t s0 = 0;  // first position of NextSet
    for (int64_t i = 0; i < n; ++i)
        if (dep[i] >= s0) {
            lp.push_back(i);
            s0 = i;
        }
    lp.push_back(n);
}

static inline int4 i4(int32_t x, int32_t y, int32_t z, int32_t w)
{
    int4 r;
    r.x = x; r.y = y; r.z = z; r.w = w;
    return r;
}

static inline int2 i2(int32_t x, int32_t y)
{
    int2 r;
    r.x = x; r.y = y;
    return r;
}

void pack_levels(const HostCSR &h, const std::vector<int32_t> &fac_graph, const std::vector<int64_t> &lp,
                 const std::vector<int32_t> &le, int max_fan, LevelPack &P)
{
    const int32_t nl = (int32_t)lp.size() - 1;
    const int T = host_threads();
    P = LevelPack{};
    auto edge_at = [&le](int64_t i) { return le.empty() ? (int32_t)i : le[i]; };
    // level and position of every scheduled edge
    std::vector<int32_t> elev(h.ne, std::numeric_limits<int32_t>::max()), pos(h.ne, -1);
    parallel_for(nl, T, 16, [&](int64_t b, int64_t e) {
        for (int64_t L = b; L < e; ++L)
            for (int64_t i = lp[L]; i < lp[L + 1]; ++i) {
                elev[edge_at(i)] = (int32_t)L;
                pos[edge_at(i)] = (int32_t)i;
            }
    });
    // A level's factors are packed in the order of their first edge in the
    // level, whole factors per warp; an edge is its factor's first in the
    // level if no other edge of the factor in the level comes earlier.
    auto first_in_level = [&](int32_t e, int32_t a, int32_t L) {
        for (int64_t q = h.fptr[a]; q < h.fptr[a + 1]; ++q)
            if (q != e && elev[q] == L && pos[q] < pos[e]) return false;
        return true;
    };
    // pass 1: lanes (whole warps) and wide-factor edges of every level
    std::vector<int64_t> lanes_at(nl + 1, 0), big_at(nl + 1, 0);
    parallel_for(nl, T, 16, [&](int64_t b, int64_t e) {
        for (int64_t L = b; L < e; ++L) {
            int64_t warps = 0, nbig = 0;
            int used = 32;
            for (int64_t i = lp[L]; i < lp[L + 1]; ++i) {
                const int32_t ed = edge_at(i), a = h.efac[ed];
                const int n = (int)(h.fptr[a + 1] - h.fptr[a]);
                if (n > max_fan) {
                    ++nbig;
                    continue;
                }
                if (!first_in_level(ed, a, (int32_t)L)) continue;
                if (used + n > 32) {
                    ++warps;
                    used = 0;
                }
                used += n;
            }
            lanes_at[L + 1] = 32 * warps;
            big_at[L + 1] = nbig;
        }
    });
    for (int32_t L = 0; L < nl; ++L) {
        P.max_lanes = std::max(P.max_lanes, (int32_t)lanes_at[L + 1]);
        lanes_at[L + 1] += lanes_at[L];
        big_at[L + 1] += big_at[L];
    }
    P.lanes.assign(lanes_at[nl], int4{-1, 0, 0, 0});
    P.lrow.assign(lanes_at[nl], int2{0, 0});
    P.big.resize(big_at[nl]);
    P.lane_ptr.resize(nl + 1);
    P.big_ptr.resize(nl + 1);
    for (int32_t L = 0; L <= nl; ++L) {
        P.lane_ptr[L] = (int32_t)lanes_at[L];
        P.big_ptr[L] = (int32_t)big_at[L];
    }
    // pass 2: fill every level at its offsets (padding lanes stay {-1, 0, 0, 0})
    parallel_for(nl, T, 16, [&](int64_t b, int64_t e) {
        for (int64_t L = b; L < e; ++L) {
            int64_t w = lanes_at[L] - 32, nb = big_at[L];  // w: first lane of the current warp
            int used = 32;
            for (int64_t i = lp[L]; i < lp[L + 1]; ++i) {
                const int32_t ed = edge_at(i), a = h.efac[ed];
                const int32_t lo = (int32_t)h.fptr[a], n = (int32_t)(h.fptr[a + 1] - h.fptr[a]);
                if (n > max_fan) {
                    P.big[nb++] = ed;
                    continue;
                }
                if (!first_in_level(ed, a, (int32_t)L)) continue;
                if (used + n > 32) {
                    w += 32;
                    used = 0;
                }
                uint32_t mask = 0;
                for (int32_t j = 0; j < n; ++j) mask |= (uint32_t)(elev[lo + j] == (int32_t)L) << j;
                int32_t pb;
                std::memcpy(&pb, &h.fparam[a], sizeof pb);
                const int32_t member = fac_graph.empty() ? 0 : fac_graph[a];
                const int32_t common = (n << 5) | ((int32_t)h.ftype[a] << 11) | (member << 15);
                for (int32_t j = 0; j < n; ++j) {
                    const int32_t v = h.fvars[lo + j];
                    P.lanes[w + used + j] = i4(lo + j, used | common | ((int32_t)((mask >> j) & 1u) << 14), pb, v);
                    P.lrow[w + used + j] = i2(h.vptr[v], h.vptr[v + 1]);
                }
                used += n;
            }
        }
    });
    P.vel.resize(h.ne);
    parallel_for(h.ne, T, 1 << 16, [&](int64_t b, int64_t e) {
        for (int64_t k = b; k < e; ++k) P.vel[k] = i2(h.vedge[k], elev[h.vedge[k]]);
    });
}

int64_t residual_classes(const HostCSR &h, const float *dres, double tol, int64_t *rank,
                         std::vector<int32_t> &act)
{
    std::vector<float> vres(h.nv, 0.f);
    for (int32_t e = 0; e < h.ne; ++e) {
        const int32_t v = h.fvars[e];
        vres[v] = std::max(vres[v], dres[e]);
    }
    act.clear();
    for (int32_t a = 0; a < h.na; ++a) {
        float rho = 0.f;
        for (int64_t q = h.fptr[a]; q < h.fptr[a + 1]; ++q) rho = std::max(rho, vres[h.fvars[q]]);
        const double r = rho;
        const int64_t c = r >= 1e-2 ? 0 : r >= 1e-4 ? 1 : r >= tol ? 2 : -1;
        for (int64_t q = h.fptr[a]; q < h.fptr[a + 1]; ++q) {
            rank[q] = c;
            if (c >= 0) act.push_back((int32_t)q);
        }
    }
    return (int64_t)act.size();
}

}  // namespace fbp
