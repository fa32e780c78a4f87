// Served form (include/fbp_serve.h): resident sessions, evidence-clamp
// requests re-run warm from the stored messages, continuous batching by a
// worker thread.
//
// Every session is one library graph on its own non-blocking stream.  A
// request is fbp_set_evidence followed by the session's own iteration (the
// flooding kernels, or one persistent level-engine launch for a static
// strategy), so its result is the plain path's result whatever else runs.
// The worker thread is the only thread that issues device work once a
// session is loaded; at every tick it
//   1. retires the chunks that finished (and queues the next chunk of a
//      request that has not stopped, or its marginals once it has),
//   2. loads waiting sessions whose memory now fits the HBM budget,
//   3. starts queued requests of idle sessions while slots are free,
//   4. frees closed sessions,
// so requests that arrive while others run join at the next tick and all
// running requests' kernels overlap on the device.
#include "fbp_serve.h"
#include "fbp_graph_impl.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <limits>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

using namespace fbp;
using Clock = std::chrono::steady_clock;

namespace {

constexpr int64_t kWarmup = -2;  // the load-time run of a session (no clamp, not reported)

struct Req {
    int32_t session = -1, var = -1;
    int8_t value = -1;
    float *result = nullptr;
    int result_dev = 0;
    Clock::time_point t_submit, t_start, t_done;
    int32_t state = FBP_REQ_QUEUED, status = 0, iters = 0;
    double residual = 0.0;
    float dev_ms = 0.f;
};

// Device memory of one session, counted byte for byte.
struct Counted {
    std::mutex mu;
    std::unordered_map<void *, size_t> size;
    int64_t bytes = 0;
};

void *counted_alloc(size_t n, void *ctx)
{
    void *p = nullptr;
    if (cudaMalloc(&p, n) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    Counted *c = static_cast<Counted *>(ctx);
    std::lock_guard<std::mutex> lock(c->mu);
    c->size[p] = n;
    c->bytes += (int64_t)n;
    return p;
}

void counted_free(void *p, void *ctx)
{
    Counted *c = static_cast<Counted *>(ctx);
    {
        std::lock_guard<std::mutex> lock(c->mu);
        auto it = c->size.find(p);
        if (it != c->size.end()) {
            c->bytes -= (int64_t)it->second;
            c->size.erase(it);
        }
    }
    cudaFree(p);
}

enum SessState { kWaiting = 0, kResident = 1, kFailed = 2, kClosed = 3 };
enum Phase { kIdle = 0, kIterating = 1, kFinishing = 2 };

struct Sess {
    int32_t id = 0;
    // the graph as opened (kept on the host until loaded)
    int32_t nv = 0, na = 0;
    std::vector<int64_t> fptr;
    std::vector<int32_t> fvars;
    std::vector<uint8_t> ftype;
    std::vector<float> fparam, prior;
    std::vector<int8_t> evidence;
    int32_t strategy = FBP_PARALL;
    std::vector<int64_t> edge_rank;
    std::vector<int32_t> factor_rank;
    bool has_edge_rank = false, has_factor_rank = false;
    int32_t residual_buckets = 0;
    int32_t max_iters = 0;
    double tol = 0.0;
    int64_t estimate = 0;
    // device state
    int state = kWaiting;
    int load_rc = FBP_OK;
    std::string load_err;
    bool closing = false;
    fbp_graph *g = nullptr;
    std::unique_ptr<Counted> mem;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_start = nullptr, ev_chunk = nullptr;
    float *h_stage = nullptr;  // pinned [nv]: marginals on their way to a host result
    // requests
    std::deque<int64_t> queue;
    int64_t cur = -1;
    int phase = kIdle;
    int32_t it_done = 0;
};

// Upper bound of a session's device bytes before it is loaded: the arrays of
// fbp_graph_create, a second message buffer, the flooding plan or the level
// plans, staging, and the per-iteration residual words.
int64_t estimate_bytes(int64_t nv, int64_t na, int64_t ne, int32_t max_iters, int strategy)
{
    int64_t b = 4 * (na + 1) + 5 * na + 16 * ne /* fvars, efac, vedge, a2v */ +
                8 * (nv + 1) /* vptr, phi */ + 4 * nv /* marginals */ + 4 * (int64_t)std::max(max_iters, 64) +
                (1 << 16);
    if (strategy == FBP_PARALL)
        b += 8 * ne /* variable-major copy, slots */ + 12 * nv /* beliefs, degree-class lists */ +
             64 * (ne / 256 + 1) /* hub chunks */;
    else
        b += 16 * ne /* the engine's row records */ + 4 * ne /* second message buffer */ +
             2 * (3 * (16 * ne + 8 * ne) / 2 + 8 * ne) /* padded lanes, rows, (edge, level) */ +
             4 * 8 * ne / 32 /* big lists, level offsets */;
    return b;
}

int64_t now_to_ms(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration_cast<std::chrono::microseconds>(b - a).count();
}

}  // namespace

struct fbp_server {
    fbp_server_config cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    std::vector<std::unique_ptr<Sess>> sess;
    std::vector<Req> req;
    int32_t inflight = 0;
    int32_t engine_owner = -1;  // session whose level-engine launch is in flight
    size_t rr = 0;              // first session considered for a free slot
    fbp_server_stats stats{};
    int64_t resident = 0;

    void run();
    bool tick();
    int load(Sess &s);
    void unload(Sess &s);
    int start(Sess &s, int64_t ticket);
    int launch_chunk(Sess &s);
    int finish_iterating(Sess &s);
    void complete(Sess &s, int status);
    void fail_request(int64_t ticket, int code);
};

namespace {

float residual_word(fbp_graph *g, cudaStream_t st, int32_t it)
{
    if (it < 1) return 0.f;
    unsigned bits = 0;
    if (cudaMemcpyAsync(&bits, g->d_res_it + (it - 1), sizeof bits, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return std::numeric_limits<float>::quiet_NaN();
    float f;
    std::memcpy(&f, &bits, sizeof f);
    return f;
}

}  // namespace

// Load a waiting session: device arrays, schedule, iteration plan; then queue
// its load-time run ahead of every request.
int fbp_server::load(Sess &s)
{
    s.mem.reset(new Counted());
    fbp_allocator alloc{counted_alloc, counted_free, s.mem.get()};
    cudaError_t e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&s.ev_start);
    if (e == cudaSuccess) e = cudaEventCreate(&s.ev_chunk);
    if (e == cudaSuccess && s.nv > 0) e = cudaMallocHost((void **)&s.h_stage, sizeof(float) * s.nv);
    if (e != cudaSuccess) return fail(FBP_ERR_CUDA, "session %d setup: %s", s.id, cudaGetErrorString(e));
    int rc = fbp_graph_create(s.nv, s.na, s.fptr.data(), s.fvars.data(), s.ftype.data(), s.fparam.data(),
                              s.prior.data(), s.evidence.data(), &alloc, s.stream, &s.g);
    if (rc) return rc;
    if (s.strategy != FBP_PARALL) {
        fbp_schedule_spec spec{s.strategy, s.has_edge_rank ? s.edge_rank.data() : nullptr,
                               s.has_factor_rank ? s.factor_rank.data() : nullptr, s.residual_buckets};
        if ((rc = fbp_schedule_set(s.g, &spec))) return rc;
    } else {
        if (!s.g->a2v_vm && (rc = dalloc_n(s.g, &s.g->a2v_vm, (size_t)s.g->h.ne))) return rc;
        if ((rc = build_flood_plan(s.g))) return rc;
    }
    if ((rc = ensure_res_cap(s.g, std::max(s.max_iters, 1)))) return rc;
    if (s.nv > 0 && !s.g->p1 && (rc = dalloc_n(s.g, &s.g->p1, (size_t)s.nv))) return rc;
    e = cudaStreamSynchronize(s.stream);
    if (e != cudaSuccess) return fail(FBP_ERR_CUDA, "session %d load: %s", s.id, cudaGetErrorString(e));
    // the host copy is no longer needed (the graph keeps its own)
    std::vector<int64_t>().swap(s.fptr);
    std::vector<int32_t>().swap(s.fvars);
    std::vector<uint8_t>().swap(s.ftype);
    std::vector<float>().swap(s.fparam);
    s.queue.push_front(kWarmup);
    return FBP_OK;
}

void fbp_server::unload(Sess &s)
{
    if (s.stream) cudaStreamSynchronize(s.stream);
    const int64_t held = s.mem ? s.mem->bytes : 0;  // what was added to `resident` at load
    if (s.g) fbp_graph_destroy(s.g);
    s.g = nullptr;
    resident -= held;
    if (s.h_stage) cudaFreeHost(s.h_stage);
    s.h_stage = nullptr;
    if (s.ev_start) cudaEventDestroy(s.ev_start);
    if (s.ev_chunk) cudaEventDestroy(s.ev_chunk);
    if (s.stream) cudaStreamDestroy(s.stream);
    s.ev_start = s.ev_chunk = nullptr;
    s.stream = nullptr;
}

// Queue the next iterations of the running request (flooding), or its one
// level-engine launch (static strategy), then a copy of the result words and
// the chunk event.
int fbp_server::launch_chunk(Sess &s)
{
    fbp_graph *g = s.g;
    if (s.strategy == FBP_PARALL) {
        // one replay of the session's captured chunk of iterations
        const int32_t k = cfg.iters_per_tick > 0 ? cfg.iters_per_tick : 16;
        if (s.max_iters > 0) {
            cudaGraphExec_t exec = nullptr;
            int rc = flood_exec_for(g, g->flood, (float)s.tol, k, &exec);
            if (rc) return rc;
            cudaError_t e = cudaGraphLaunch(exec, s.stream);
            if (e != cudaSuccess) return fail(FBP_ERR_CUDA, "chunk: %s", cudaGetErrorString(e));
            stats.kernel_launches += (int64_t)k * flood_launches(g->d, g->flood);
        }
        s.it_done = std::min(s.max_iters, s.it_done + k);
    } else if (s.max_iters > 0) {
        EngineArgs A = engine_args(g);
        A.res = g->d_res_it;
        A.max_iters = s.max_iters;
        A.tol = (float)s.tol;
        int grid = 1, cluster = 0;
        engine_shape(g, &grid, &cluster);
        cudaError_t e = launch_engine(A, grid, cluster, s.stream);
        if (e != cudaSuccess) return fail(FBP_ERR_CUDA, "engine launch: %s", cudaGetErrorString(e));
        stats.kernel_launches += 1;
        engine_owner = s.id;
        s.it_done = s.max_iters;
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->h_out, g->d_out, sizeof(int32_t) * 4, cudaMemcpyDeviceToHost, s.stream);
    if (e == cudaSuccess) e = cudaEventRecord(s.ev_chunk, s.stream);
    if (e != cudaSuccess) return fail(FBP_ERR_CUDA, "chunk: %s", cudaGetErrorString(e));
    return FBP_OK;
}

// Begin a request (or the load-time run): clamp, clear the run's words, queue
// the first chunk.
int fbp_server::start(Sess &s, int64_t ticket)
{
    fbp_graph *g = s.g;
    int rc = FBP_OK;
    if (ticket != kWarmup) {
        Req &r = req[ticket];
        if ((rc = fbp_set_evidence(g, r.var, r.value))) return rc;
        r.state = FBP_REQ_RUNNING;
        r.t_start = Clock::now();
    }
    cudaError_t e = cudaEventRecord(s.ev_start, s.stream);
    g->h_out[0] = g->h_out[1] = g->h_out[2] = 0;
    g->h_out[3] = s.max_iters;  // the flooding kernels' iteration limit
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->d_out, g->h_out, sizeof(int32_t) * 4, cudaMemcpyHostToDevice, s.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->d_guards, 0, sizeof(unsigned long long), s.stream);
    if (s.strategy == FBP_PARALL) {
        if (e == cudaSuccess) e = cudaMemsetAsync(g->d_res, 0, sizeof(unsigned) * kResSlots, s.stream);
        if (e == cudaSuccess) {
            flood_sync(g->d, g->a2v[g->cur], g->a2v_vm, s.stream);
            stats.kernel_launches += g->h.ne > 0;
        }
    } else {
        if (e == cudaSuccess)
            e = cudaMemsetAsync(g->d_res_it, 0, sizeof(unsigned) * std::max(s.max_iters, 1), s.stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(g->d_bar, 0, sizeof(unsigned) * 2, s.stream);
    }
    if (e != cudaSuccess) return fail(FBP_ERR_CUDA, "request start: %s", cudaGetErrorString(e));
    s.cur = ticket;
    s.it_done = 0;
    s.phase = kIterating;
    ++inflight;
    stats.peak_inflight = std::max(stats.peak_inflight, inflight);
    return launch_chunk(s);
}

// The run has stopped: its iteration count, residual and (if asked for) the
// marginals on their way to the caller's buffer.
int fbp_server::finish_iterating(Sess &s)
{
    fbp_graph *g = s.g;
    int32_t it = 0;
    int status = FBP_NOT_CONVERGED;
    if (s.strategy == FBP_PARALL) {
        it = s.max_iters == 0 ? 0 : g->h_out[1];
        status = g->h_out[0] == 1 ? FBP_OK : FBP_NOT_CONVERGED;
    } else if (s.max_iters > 0) {
        if (engine_owner == s.id) engine_owner = -1;
        if (g->h_out[2]) return fail(FBP_ERR_TIMEOUT, "a device-side barrier wait expired");
        it = g->h_out[0];
        status = g->h_out[1] == 0 ? FBP_OK : FBP_NOT_CONVERGED;
        g->cur ^= (it * (int32_t)g->halves.size()) & 1;
    }
    const float res = residual_word(g, s.stream, it);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, s.ev_start, s.ev_chunk);
    if (s.cur == kWarmup) {
        s.phase = kIdle;
        s.cur = -1;
        --inflight;
        return FBP_OK;
    }
    Req &r = req[s.cur];
    r.iters = it;
    r.status = status;
    r.residual = (double)res;
    r.dev_ms = ms;
    if (r.result && s.nv > 0) {
        float *dst = r.result_dev ? r.result : g->p1;
        if (int rc = marginals_launch(g, dst, s.stream)) return rc;
        stats.kernel_launches += 1 + (g->n_marg_rows > 0);
        cudaError_t e = cudaSuccess;
        if (e == cudaSuccess && !r.result_dev)
            e = cudaMemcpyAsync(s.h_stage, g->p1, sizeof(float) * s.nv, cudaMemcpyDeviceToHost, s.stream);
        if (e == cudaSuccess) e = cudaEventRecord(s.ev_chunk, s.stream);
        if (e != cudaSuccess) return fail(FBP_ERR_CUDA, "marginals: %s", cudaGetErrorString(e));
    } else {
        cudaEventRecord(s.ev_chunk, s.stream);
    }
    s.phase = kFinishing;
    return FBP_OK;
}

void fbp_server::complete(Sess &s, int status)
{
    Req &r = req[s.cur];
    if (r.result && !r.result_dev && s.nv > 0) std::memcpy(r.result, s.h_stage, sizeof(float) * s.nv);
    r.t_done = Clock::now();
    r.state = status < 0 ? FBP_REQ_FAILED : FBP_REQ_DONE;
    if (status < 0) r.status = status;
    if (status < 0) ++stats.failed;
    else ++stats.completed;
    s.phase = kIdle;
    s.cur = -1;
    --inflight;
    cv_done.notify_all();
}

void fbp_server::fail_request(int64_t ticket, int code)
{
    if (ticket == kWarmup) return;
    Req &r = req[ticket];
    r.state = FBP_REQ_FAILED;
    r.status = code;
    r.t_done = Clock::now();
    ++stats.failed;
    cv_done.notify_all();
}

// One pass of the scheduler; true if it changed anything.
bool fbp_server::tick()
{
    bool busy = false, launched = false;
    // 1. retire finished chunks
    for (auto &sp : sess) {
        Sess &s = *sp;
        if (s.state != kResident || s.phase == kIdle) continue;
        cudaError_t q = cudaEventQuery(s.ev_chunk);
        if (q == cudaErrorNotReady) continue;
        busy = true;
        int rc = q == cudaSuccess ? FBP_OK : fail(FBP_ERR_CUDA, "session %d: %s", s.id, cudaGetErrorString(q));
        if (!rc && s.phase == kIterating) {
            const bool stopped = s.strategy != FBP_PARALL || s.g->h_out[0] != 0 || s.it_done >= s.max_iters;
            if (!stopped) {
                rc = launch_chunk(s);
                launched = true;
            } else {
                rc = finish_iterating(s);
            }
            if (!rc) continue;
        } else if (!rc && s.phase == kFinishing) {
            complete(s, FBP_OK);
            continue;
        }
        // a failed step fails the request; the session stays usable
        if (s.cur == kWarmup) {
            s.phase = kIdle;
            s.cur = -1;
            --inflight;
        } else if (s.cur >= 0) {
            const int64_t t = s.cur;
            s.phase = kIdle;
            s.cur = -1;
            --inflight;
            fail_request(t, rc);
        }
        if (engine_owner == s.id) engine_owner = -1;
    }
    // 2. load waiting sessions that fit the budget, in the order they were opened
    for (auto &sp : sess) {
        Sess &s = *sp;
        if (s.state != kWaiting) continue;
        if (s.closing) {
            s.state = kClosed;
            while (!s.queue.empty()) fail_request(s.queue.front(), FBP_ERR_INVALID_ARG), s.queue.pop_front();
            cv_done.notify_all();
            continue;
        }
        if (cfg.hbm_budget_bytes > 0 && resident + s.estimate > cfg.hbm_budget_bytes) break;
        busy = true;
        int rc = load(s);
        if (s.mem) resident += s.mem->bytes;
        stats.peak_resident_bytes = std::max(stats.peak_resident_bytes, resident);
        if (rc) {
            s.state = kFailed;
            s.load_rc = rc;
            s.load_err = fbp_last_error();
            unload(s);
            while (!s.queue.empty()) {
                const int64_t t = s.queue.front();
                s.queue.pop_front();
                fail_request(t, rc);
            }
        } else {
            s.state = kResident;
        }
        cv_done.notify_all();
    }
    // 3. start queued requests of idle sessions while slots are free, taking
    //    the sessions round-robin so that none is starved of slots
    const int32_t slots = cfg.max_inflight > 0 ? cfg.max_inflight : 64;
    const size_t ns = sess.size();
    for (size_t k = 0; k < ns; ++k) {
        Sess &s = *sess[(rr + k) % ns];
        if (inflight >= slots) {
            rr = (rr + k) % ns;
            break;
        }
        if (s.state != kResident || s.phase != kIdle || s.queue.empty()) continue;
        if (s.strategy != FBP_PARALL && engine_owner >= 0) continue;  // one grid-wide engine at a time
        const int64_t t = s.queue.front();
        s.queue.pop_front();
        busy = launched = true;
        int rc = start(s, t);
        if (rc) {
            if (s.phase != kIdle) {
                s.phase = kIdle;
                s.cur = -1;
                --inflight;
            }
            if (engine_owner == s.id) engine_owner = -1;
            fail_request(t, rc);
        }
    }
    // 4. free closed sessions
    for (auto &sp : sess) {
        Sess &s = *sp;
        if (!s.closing || s.state != kResident || s.phase != kIdle || !s.queue.empty()) continue;
        unload(s);
        s.state = kClosed;
        busy = true;
        cv_done.notify_all();
    }
    if (launched) ++stats.ticks;
    return busy;
}

void fbp_server::run()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lock(mu);
    int idle = 0;
    for (;;) {
        if (stop) {
            // nothing new starts: queued requests were failed by the caller;
            // sessions still waiting for memory are dropped
            for (auto &sp : sess)
                if (sp->state == kWaiting) sp->state = kClosed;
        }
        const bool busy = tick();
        if (stop && inflight == 0) break;
        if (busy) {
            idle = 0;
            continue;
        }
        if (inflight > 0) {
            // chunks in flight: poll again soon
            lock.unlock();
            if (++idle < 64) std::this_thread::yield();
            else std::this_thread::sleep_for(std::chrono::microseconds(20));
            lock.lock();
        } else {
            idle = 0;
            cv_work.wait_for(lock, std::chrono::milliseconds(50));
        }
    }
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" int fbp_server_create(const fbp_server_config *cfg, fbp_server **out)
{
    if (!out) return fail(FBP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    fbp_server_config c{};
    if (cfg) c = *cfg;
    if (c.hbm_budget_bytes < 0 || c.max_inflight < 0 || c.iters_per_tick < 0)
        return fail(FBP_ERR_INVALID_ARG, "negative configuration field");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(FBP_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    fbp_server *s = new fbp_server();
    s->cfg = c;
    s->device = dev;
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return FBP_OK;
}

extern "C" int fbp_server_session_open(fbp_server *srv, const fbp_graph_desc *d, int32_t *session_out)
{
    if (!srv || !d || !session_out) return fail(FBP_ERR_INVALID_ARG, "NULL argument");
    int rc = check_graph_args(d->n_vars, d->n_factors, d->factor_ptr, d->factor_vars, d->factor_type,
                              d->factor_param, d->prior_p1, d->evidence);
    if (rc) return rc;
    const int st = d->schedule.strategy;
    if (st < FBP_PARALL || st > FBP_CUSTOM_RANK || st == FBP_RESIDUAL)
        return fail(FBP_ERR_INVALID_ARG, "session strategy %d is not PARALL or a static strategy", st);
    if (d->max_iters < 0 || !(d->tol >= 0.0)) return fail(FBP_ERR_INVALID_ARG, "bad max_iters or tol");
    for (int32_t a = 0; a < d->n_factors; ++a)
        if (d->factor_type[a] == FBP_TERMS)
            return fail(FBP_ERR_INVALID_ARG, "generic (FBP_TERMS) factors are for single graphs");
    const int64_t ne = d->factor_ptr[d->n_factors];
    if (ne >= ((int64_t)1 << 31)) return fail(FBP_ERR_INVALID_ARG, "graph too large");
    std::unique_ptr<Sess> s(new Sess());
    s->nv = d->n_vars;
    s->na = d->n_factors;
    s->fptr.assign(d->factor_ptr, d->factor_ptr + d->n_factors + 1);
    s->fvars.assign(d->factor_vars, d->factor_vars + ne);
    s->ftype.assign(d->factor_type, d->factor_type + d->n_factors);
    s->fparam.assign(d->factor_param, d->factor_param + d->n_factors);
    if (d->prior_p1) s->prior.assign(d->prior_p1, d->prior_p1 + d->n_vars);
    else s->prior.assign(d->n_vars, std::numeric_limits<float>::quiet_NaN());
    if (d->evidence) s->evidence.assign(d->evidence, d->evidence + d->n_vars);
    else s->evidence.assign(d->n_vars, (int8_t)-1);
    s->strategy = st;
    if (d->schedule.edge_rank) s->edge_rank.assign(d->schedule.edge_rank, d->schedule.edge_rank + ne), s->has_edge_rank = true;
    if (d->schedule.factor_rank)
        s->factor_rank.assign(d->schedule.factor_rank, d->schedule.factor_rank + d->n_factors), s->has_factor_rank = true;
    s->residual_buckets = d->schedule.residual_buckets;
    s->max_iters = d->max_iters;
    s->tol = d->tol;
    s->estimate = estimate_bytes(d->n_vars, d->n_factors, ne, d->max_iters, st);
    if (srv->cfg.hbm_budget_bytes > 0 && s->estimate > srv->cfg.hbm_budget_bytes)
        return fail(FBP_ERR_INVALID_ARG, "session needs about %lld bytes, more than the whole budget (%lld)",
                    (long long)s->estimate, (long long)srv->cfg.hbm_budget_bytes);
    std::unique_lock<std::mutex> lock(srv->mu);
    const int32_t id = (int32_t)srv->sess.size();
    s->id = id;
    const bool fits_now = srv->cfg.hbm_budget_bytes == 0 ||
                          srv->resident + s->estimate <= srv->cfg.hbm_budget_bytes;
    bool ahead = false;  // an earlier session still waits for memory: this one queues behind it
    for (auto &sp : srv->sess) ahead = ahead || sp->state == kWaiting;
    srv->sess.push_back(std::move(s));
    Sess &ref = *srv->sess.back();
    srv->cv_work.notify_all();
    *session_out = id;
    if (!fits_now || ahead) return FBP_OK;  // loads once memory is free
    srv->cv_done.wait(lock, [&] { return ref.state != kWaiting; });
    if (ref.state == kFailed) return fail(ref.load_rc, "%s", ref.load_err.c_str());
    return FBP_OK;
}

extern "C" int fbp_server_session_close(fbp_server *srv, int32_t session)
{
    if (!srv) return fail(FBP_ERR_INVALID_ARG, "NULL argument");
    std::unique_lock<std::mutex> lock(srv->mu);
    if (session < 0 || session >= (int32_t)srv->sess.size()) return fail(FBP_ERR_INVALID_ARG, "unknown session");
    Sess &s = *srv->sess[session];
    if (s.state == kClosed) return FBP_OK;
    s.closing = true;
    if (s.state == kFailed) {
        s.state = kClosed;
        return FBP_OK;
    }
    srv->cv_work.notify_all();
    srv->cv_done.wait(lock, [&] { return s.state == kClosed || s.state == kFailed; });
    return FBP_OK;
}

extern "C" int fbp_server_submit(fbp_server *srv, int32_t session, int32_t var, int8_t value, float *result_p1,
                                 int result_is_device, int64_t *ticket_out)
{
    if (!srv || !ticket_out) return fail(FBP_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lock(srv->mu);
    if (session < 0 || session >= (int32_t)srv->sess.size()) return fail(FBP_ERR_INVALID_ARG, "unknown session");
    Sess &s = *srv->sess[session];
    if (s.closing || s.state == kClosed || s.state == kFailed)
        return fail(FBP_ERR_INVALID_ARG, "session %d is closed or failed to load", session);
    if (var < 0 || var >= s.nv) return fail(FBP_ERR_INVALID_ARG, "variable %d out of range", var);
    if (value < -1 || value > 1) return fail(FBP_ERR_INVALID_ARG, "value must be -1, 0 or 1");
    Req r;
    r.session = session;
    r.var = var;
    r.value = value;
    r.result = result_p1;
    r.result_dev = result_is_device;
    r.t_submit = Clock::now();
    const int64_t t = (int64_t)srv->req.size();
    srv->req.push_back(r);
    s.queue.push_back(t);
    ++srv->stats.submitted;
    *ticket_out = t;
    srv->cv_work.notify_all();
    return FBP_OK;
}

namespace {
void fill_info(const fbp_server *srv, int64_t t, fbp_request_info *info)
{
    const Req &r = srv->req[t];
    info->state = r.state;
    info->status = r.status;
    info->iters = r.iters;
    info->session = r.session;
    info->residual = r.residual;
    const bool started = r.state != FBP_REQ_QUEUED;
    const bool done = r.state == FBP_REQ_DONE || r.state == FBP_REQ_FAILED;
    info->queue_ms = started && r.t_start.time_since_epoch().count() ? now_to_ms(r.t_submit, r.t_start) / 1e3 : 0.0;
    info->latency_ms = done ? now_to_ms(r.t_submit, r.t_done) / 1e3 : 0.0;
    info->device_ms = r.dev_ms;
}
}  // namespace

extern "C" int fbp_server_poll(fbp_server *srv, int64_t ticket, fbp_request_info *info)
{
    if (!srv || !info) return fail(FBP_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lock(srv->mu);
    if (ticket < 0 || ticket >= (int64_t)srv->req.size()) return fail(FBP_ERR_INVALID_ARG, "unknown ticket");
    fill_info(srv, ticket, info);
    return FBP_OK;
}

extern "C" int fbp_server_wait(fbp_server *srv, int64_t ticket, fbp_request_info *info)
{
    if (!srv) return fail(FBP_ERR_INVALID_ARG, "NULL argument");
    std::unique_lock<std::mutex> lock(srv->mu);
    if (ticket < 0 || ticket >= (int64_t)srv->req.size()) return fail(FBP_ERR_INVALID_ARG, "unknown ticket");
    srv->cv_done.wait(lock, [&] {
        const int st = srv->req[ticket].state;
        return st == FBP_REQ_DONE || st == FBP_REQ_FAILED;
    });
    if (info) fill_info(srv, ticket, info);
    return FBP_OK;
}

extern "C" int fbp_server_drain(fbp_server *srv)
{
    if (!srv) return fail(FBP_ERR_INVALID_ARG, "NULL argument");
    std::unique_lock<std::mutex> lock(srv->mu);
    srv->cv_done.wait(lock, [&] { return srv->stats.completed + srv->stats.failed == srv->stats.submitted; });
    return FBP_OK;
}

extern "C" int fbp_server_get_stats(fbp_server *srv, fbp_server_stats *out)
{
    if (!srv || !out) return fail(FBP_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lock(srv->mu);
    *out = srv->stats;
    out->resident_bytes = srv->resident;
    out->sessions_resident = out->sessions_waiting = out->sessions_warming = 0;
    for (auto &sp : srv->sess) {
        out->sessions_resident += sp->state == kResident;
        out->sessions_waiting += sp->state == kWaiting;
        out->sessions_warming += sp->state == kResident &&
                                 (sp->cur == kWarmup || (!sp->queue.empty() && sp->queue.front() == kWarmup));
    }
    return FBP_OK;
}

extern "C" void fbp_server_destroy(fbp_server *srv)
{
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        // queued requests fail; running ones finish
        for (auto &sp : srv->sess) {
            while (!sp->queue.empty()) {
                const int64_t t = sp->queue.front();
                sp->queue.pop_front();
                srv->fail_request(t, FBP_ERR_INVALID_ARG);
            }
        }
        srv->stop = true;
        srv->cv_work.notify_all();
    }
    if (srv->worker.joinable()) srv->worker.join();
    cudaSetDevice(srv->device);
    for (auto &sp : srv->sess)
        if (sp->state == kResident) srv->unload(*sp);
    delete srv;
}
