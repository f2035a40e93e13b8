// nls_serve.cu -- continuous-batching request server over the batched solver.
//
// Clients submit solve requests (a batch of instances of one family and n,
// on HOST buffers) at any time.  A dispatcher thread admits waiting
// requests in arrival order as soon as their state fits in the device
// arena -- the admission test is free device memory -- copies their inputs
// to the device, and flushes each wave of admitted requests through one of
// several worker handles, each on its own stream, so waves that arrive
// while others are still running overlap on the GPU.  When a request's
// results are back on the host its arena space is released and the next
// waiting requests are admitted.  All solver work runs in the library's
// kernels; this file only schedules, copies and times.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/nls.h"
#include "nls_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over one device arena (offsets, 256-byte aligned).
struct Arena {
    size_t size = 0;
    std::map<size_t, size_t> free_; // offset -> length
    void reset(size_t n)
    {
        size = n;
        free_.clear();
        free_[0] = n;
    }
    bool alloc(size_t n, size_t *off)
    {
        n = (n + 255) & ~size_t(255);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n, at = it->first + n;
                free_.erase(it);
                if (rest) free_[at] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n)
    {
        n = (n + 255) & ~size_t(255);
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t largest() const
    {
        size_t m = 0;
        for (auto &kv : free_) m = std::max(m, kv.second);
        return m;
    }
};

// Timing events of one worker wave: before its input copies, before its
// solve launch, after it.
struct WaveEvents {
    cudaEvent_t a = nullptr, b = nullptr, c = nullptr;
    bool ok = false;
    WaveEvents()
    {
        ok = cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess &&
             cudaEventCreate(&c) == cudaSuccess;
    }
    ~WaveEvents()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
        if (c) cudaEventDestroy(c);
    }
};

struct Ticket {
    int64_t id = 0;
    int family = 0, n = 0, alg = 0, maxiters = 0;
    double abstol = 0.0;
    int64_t batch = 0;
    const double *h_params = nullptr;
    double *h_u = nullptr;
    nls_outputs h_out{};
    size_t bytes = 0, off = 0;
    int worker = -1;
    int64_t req = 0;
    cudaEvent_t ev = nullptr;
    double t_submit = 0.0, t_admit = 0.0, t_launch = 0.0, t_done = 0.0;
    std::shared_ptr<WaveEvents> wave;
    float h2d_ms = -1.f, solve_ms = -1.f, d2h_ms = -1.f;
    int wave_requests = 0;
    int64_t solved = -1;
    int state = 0; // 0 queued, 1 in flight, 2 done, 3 failed
    bool failed = false; // enqueueing failed; state becomes 3 once its copies are done
    std::string err;
};

} // namespace

struct nls_server {
    int device = 0;
    Clock::time_point t0;
    std::vector<nls_handle> workers;
    std::vector<cudaStream_t> streams;
    std::vector<int> load;      // in-flight tickets per worker
    char *arena_d = nullptr;
    Arena arena;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Ticket>> queue;
    std::map<int64_t, std::shared_ptr<Ticket>> tickets;
    std::vector<std::shared_ptr<Ticket>> inflight;
    int64_t next_id = 1;
    std::atomic<bool> stop{false};
    std::thread thr;
    std::string fatal;
    // statistics
    int64_t admitted = 0, completed = 0, solved = 0, max_queue = 0, max_inflight = 0, waves = 0;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

static std::mutex g_serr_mu;
static std::string g_serr;

static int serr(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    std::lock_guard<std::mutex> g(g_serr_mu);
    g_serr = buf;
    return nls::set_global_error(code, buf);
}

static size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

static size_t n_params(int family, int n)
{
    return family == NLS_CUBIC ? size_t(n) * n + n : family == NLS_BRATU ? 1 : family == NLS_SQUARE ? n : 0;
}

static size_t ticket_bytes(int family, int n, int64_t batch)
{
    return al256(n_params(family, n) * batch * 8) + al256(size_t(n) * batch * 8) + al256(batch * 8) +
           4 * al256(batch * 4);
}

// Device layout of a ticket's arena block: params, u, resid, status, iters, nfev, ngrad.
struct Layout {
    double *p, *u, *resid;
    int32_t *status, *iters, *nfev, *ngrad;
};

static Layout layout(const Ticket &t, char *arena)
{
    const size_t E = n_params(t.family, t.n);
    Layout L;
    char *c = arena + t.off;
    L.p = reinterpret_cast<double *>(c);
    c += al256(E * t.batch * 8);
    L.u = reinterpret_cast<double *>(c);
    c += al256(size_t(t.n) * t.batch * 8);
    L.resid = reinterpret_cast<double *>(c);
    c += al256(t.batch * 8);
    L.status = reinterpret_cast<int32_t *>(c);
    c += al256(t.batch * 4);
    L.iters = reinterpret_cast<int32_t *>(c);
    c += al256(t.batch * 4);
    L.nfev = reinterpret_cast<int32_t *>(c);
    c += al256(t.batch * 4);
    L.ngrad = reinterpret_cast<int32_t *>(c);
    return L;
}

// Dispatcher: admit, launch, retire.  Runs until stop is set and all
// admitted work has retired.
static void dispatcher(nls_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    int idle_polls = 0;
    for (;;) {
        // ---- admit waiting requests in arrival order while they fit
        std::vector<std::vector<std::shared_ptr<Ticket>>> wave(s->workers.size());
        while (!s->queue.empty()) {
            auto t = s->queue.front();
            size_t off = 0;
            if (!s->arena.alloc(t->bytes, &off)) break;
            s->queue.pop_front();
            t->off = off;
            int w = 0;
            for (int i = 1; i < (int)s->workers.size(); ++i)
                if (s->load[i] < s->load[w]) w = i;
            t->worker = w;
            ++s->load[w];
            t->t_admit = s->now();
            t->state = 1;
            ++s->admitted;
            wave[w].push_back(t);
        }
        lk.unlock();
        // ---- copy inputs, enqueue and flush each worker's wave
        for (size_t w = 0; w < wave.size(); ++w) {
            if (wave[w].empty()) continue;
            nls_handle h = s->workers[w];
            cudaStream_t st = s->streams[w];
            auto W = std::make_shared<WaveEvents>();
            // all of the wave's input copies first, back to back on the stream;
            // then the requests are enqueued (host work only until the flush)
            if (W->ok) cudaEventRecord(W->a, st);
            for (auto &t : wave[w]) {
                const size_t E = n_params(t->family, t->n);
                const Layout L = layout(*t, s->arena_d);
                cudaError_t e = cudaSuccess;
                if (E && t->batch) e = cudaMemcpyAsync(L.p, t->h_params, E * t->batch * 8, cudaMemcpyHostToDevice, st);
                if (e == cudaSuccess && t->batch)
                    e = cudaMemcpyAsync(L.u, t->h_u, size_t(t->n) * t->batch * 8, cudaMemcpyHostToDevice, st);
                if (e != cudaSuccess) {
                    t->failed = true;
                    t->err = cudaGetErrorString(e);
                }
            }
            if (W->ok) cudaEventRecord(W->b, st);
            for (auto &t : wave[w]) {
                if (t->failed) continue;
                const size_t E = n_params(t->family, t->n);
                const Layout L = layout(*t, s->arena_d);
                nls_outputs dout{L.status, L.iters, L.resid, L.nfev, L.ngrad};
                if (nls_solve(h, t->family, E ? L.p : nullptr, L.u, t->n, t->batch, t->alg, t->abstol, t->maxiters,
                              &dout, &t->req)) {
                    t->failed = true;
                    t->err = nls_last_error(h);
                }
            }
            nls_flush(h);
            if (W->ok) cudaEventRecord(W->c, st);
            const double t_launch = s->now();
            for (auto &t : wave[w]) {
                t->t_launch = t_launch;
                t->wave_requests = (int)wave[w].size();
                if (W->ok) t->wave = W;
                if (t->failed) {
                    // its input copies may already be queued on the stream: the
                    // arena block is released only once the stream has passed them
                    if (cudaEventCreateWithFlags(&t->ev, cudaEventDisableTiming) != cudaSuccess ||
                        cudaEventRecord(t->ev, st) != cudaSuccess) {
                        if (t->ev) cudaEventDestroy(t->ev);
                        t->ev = nullptr;
                        cudaStreamSynchronize(st);
                    }
                    continue;
                }
                const Layout L = layout(*t, s->arena_d);
                if (t->batch) {
                    cudaMemcpyAsync(t->h_u, L.u, size_t(t->n) * t->batch * 8, cudaMemcpyDeviceToHost, st);
                    if (t->h_out.status) cudaMemcpyAsync(t->h_out.status, L.status, t->batch * 4, cudaMemcpyDeviceToHost, st);
                    if (t->h_out.iters) cudaMemcpyAsync(t->h_out.iters, L.iters, t->batch * 4, cudaMemcpyDeviceToHost, st);
                    if (t->h_out.nfev) cudaMemcpyAsync(t->h_out.nfev, L.nfev, t->batch * 4, cudaMemcpyDeviceToHost, st);
                    if (t->h_out.ngrad)
                        cudaMemcpyAsync(t->h_out.ngrad, L.ngrad, t->batch * 4, cudaMemcpyDeviceToHost, st);
                    if (t->h_out.resid_inf)
                        cudaMemcpyAsync(t->h_out.resid_inf, L.resid, t->batch * 8, cudaMemcpyDeviceToHost, st);
                }
                if (t->wave) cudaEventCreate(&t->ev); // timed: the wave's events are its base
                else cudaEventCreateWithFlags(&t->ev, cudaEventDisableTiming);
                cudaEventRecord(t->ev, st);
            }
        }
        lk.lock();
        bool retire_failed = false;
        for (size_t w = 0; w < wave.size(); ++w) {
            if (!wave[w].empty()) ++s->waves;
            for (auto &t : wave[w]) {
                if (t->failed && !t->ev) { // the stream was synchronised above
                    s->arena.release(t->off, t->bytes);
                    --s->load[t->worker];
                    t->t_done = s->now();
                    t->state = 3;
                    retire_failed = true;
                    continue;
                }
                s->inflight.push_back(t);
            }
        }
        s->max_inflight = std::max<int64_t>(s->max_inflight, (int64_t)s->inflight.size());
        // ---- retire completed requests (and failed ones whose copies are done)
        bool retired = retire_failed;
        for (size_t i = 0; i < s->inflight.size();) {
            auto t = s->inflight[i];
            if (cudaEventQuery(t->ev) == cudaSuccess) {
                if (t->wave && !t->failed) {
                    cudaEventElapsedTime(&t->h2d_ms, t->wave->a, t->wave->b);
                    cudaEventElapsedTime(&t->solve_ms, t->wave->b, t->wave->c);
                    cudaEventElapsedTime(&t->d2h_ms, t->wave->c, t->ev);
                }
                t->wave.reset();
                cudaEventDestroy(t->ev);
                t->ev = nullptr;
                t->t_done = s->now();
                s->arena.release(t->off, t->bytes);
                --s->load[t->worker];
                if (t->failed) {
                    t->state = 3;
                } else {
                    int64_t sv = -1;
                    nls_status(s->workers[t->worker], t->req, &sv, 0);
                    t->solved = sv;
                    t->state = 2;
                    ++s->completed;
                    s->solved += std::max<int64_t>(sv, 0);
                }
                s->inflight[i] = s->inflight.back();
                s->inflight.pop_back();
                retired = true;
            } else {
                ++i;
            }
        }
        if (retired) s->cv_done.notify_all();
        if (s->stop && s->queue.empty() && s->inflight.empty()) break;
        if (s->inflight.empty() && s->queue.empty()) {
            s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
            idle_polls = 0;
        } else if (!retired) {
            // poll completions while work is in flight: yield (a few microseconds
            // per round) for the first ~2000 rounds after the last completion,
            // then 20 us sleeps (which the kernel's timer slack stretches to
            // 60-80 us), so a long solve does not keep a core spinning
            lk.unlock();
            if (++idle_polls < 2000) std::this_thread::yield();
            else std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        } else {
            idle_polls = 0;
        }
    }
}

extern "C" {

int nls_server_create(nls_server_t *out, int device, size_t mem_budget_bytes, int streams)
{
    if (!out) return serr(NLS_E_INVALID, "out is NULL");
    *out = nullptr;
    if (streams < 1 || streams > 16) return serr(NLS_E_INVALID, "streams = %d outside 1..16", streams);
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return serr(NLS_E_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    size_t free_b = 0, total_b = 0;
    e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) return serr(NLS_E_CUDA, "cudaMemGetInfo: %s", cudaGetErrorString(e));
    // admission budget: the requested bytes, never more than free memory minus 1 GiB
    const size_t reserve = size_t(1) << 30;
    size_t budget = mem_budget_bytes ? mem_budget_bytes : (free_b > 2 * reserve ? free_b / 2 : free_b / 4);
    if (free_b > reserve) budget = std::min(budget, free_b - reserve);
    std::unique_ptr<nls_server> s(new nls_server);
    s->device = device;
    s->t0 = Clock::now();
    e = cudaMalloc((void **)&s->arena_d, budget);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return serr(NLS_E_NOMEM, "arena of %zu bytes: %s", budget, cudaGetErrorString(e));
    }
    s->arena.reset(budget);
    for (int i = 0; i < streams; ++i) {
        cudaStream_t st;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) return serr(NLS_E_CUDA, "stream: %s", cudaGetErrorString(e));
        nls_handle h = nullptr;
        int rc = nls_batch_create(&h, device, st, 0);
        if (rc) return rc;
        s->streams.push_back(st);
        s->workers.push_back(h);
        s->load.push_back(0);
    }
    nls_server *raw = s.release();
    raw->thr = std::thread(dispatcher, raw);
    *out = raw;
    return NLS_OK;
}

int nls_server_submit(nls_server_t s, int family, const double *params, double *u, int n, int64_t batch, int alg,
                      double abstol, int maxiters, const nls_outputs *out, int64_t *ticket)
{
    if (!s || !ticket) return serr(NLS_E_INVALID, "NULL server or ticket");
    if (family < 0 || family > NLS_ROSENBROCK) return serr(NLS_E_UNSUPPORTED, "unknown family %d", family);
    if (n < 1 || n > 128) return serr(NLS_E_UNSUPPORTED, "n = %d outside [1, 128]", n);
    if (batch < 0 || maxiters < 0 || !(abstol >= 0.0)) return serr(NLS_E_INVALID, "bad batch / maxiters / abstol");
    if (batch > 0 && (!u || (family != NLS_ROSENBROCK && !params))) return serr(NLS_E_INVALID, "NULL params or u");
    auto t = std::make_shared<Ticket>();
    t->family = family;
    t->n = n;
    t->batch = batch;
    t->alg = alg;
    t->abstol = abstol;
    t->maxiters = maxiters;
    t->h_params = params;
    t->h_u = u;
    if (out) t->h_out = *out;
    t->bytes = ticket_bytes(family, n, batch);
    std::lock_guard<std::mutex> g(s->mu);
    if (t->bytes > s->arena.size)
        return serr(NLS_E_NOMEM, "request needs %zu bytes, the arena holds %zu", t->bytes, s->arena.size);
    t->id = s->next_id++;
    t->t_submit = s->now();
    s->tickets[t->id] = t;
    s->queue.push_back(t);
    s->max_queue = std::max<int64_t>(s->max_queue, (int64_t)s->queue.size());
    *ticket = t->id;
    s->cv_work.notify_one();
    return NLS_OK;
}

int nls_server_wait_timed(nls_server_t s, int64_t ticket, int64_t *solved, nls_server_timing *timing,
                          int timeout_ms)
{
    if (!s) return serr(NLS_E_INVALID, "NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return serr(NLS_E_NOTFOUND, "unknown ticket %lld", (long long)ticket);
    auto t = it->second;
    auto done = [&] { return t->state >= 2; };
    if (timeout_ms < 0) s->cv_done.wait(lk, done);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done))
        return serr(NLS_E_TIMEOUT, "ticket %lld not complete", (long long)ticket);
    s->tickets.erase(it);
    if (t->state == 3) return serr(NLS_E_CUDA, "ticket %lld failed: %s", (long long)ticket, t->err.c_str());
    if (solved) *solved = t->solved;
    if (timing) {
        timing->t_submit = t->t_submit;
        timing->t_admit = t->t_admit;
        timing->t_launch = t->t_launch;
        timing->t_done = t->t_done;
        timing->h2d_ms = t->h2d_ms;
        timing->solve_ms = t->solve_ms;
        timing->d2h_ms = t->d2h_ms;
        timing->wave_requests = t->wave_requests;
    }
    return NLS_OK;
}

int nls_server_wait(nls_server_t s, int64_t ticket, int64_t *solved, double *t_submit, double *t_done,
                    int timeout_ms)
{
    nls_server_timing tm{};
    const int rc = nls_server_wait_timed(s, ticket, solved, &tm, timeout_ms);
    if (rc == NLS_OK) {
        if (t_submit) *t_submit = tm.t_submit;
        if (t_done) *t_done = tm.t_done;
    }
    return rc;
}

double nls_server_now(nls_server_t s) { return s ? s->now() : 0.0; }

int nls_server_stats(nls_server_t s, int64_t *counters, int ncounters)
{
    if (!s || !counters) return serr(NLS_E_INVALID, "NULL argument");
    std::lock_guard<std::mutex> g(s->mu);
    const int64_t v[] = {s->admitted, s->completed, s->solved, s->max_queue, s->max_inflight, s->waves,
                         (int64_t)s->queue.size(), (int64_t)s->inflight.size(), (int64_t)s->arena.size,
                         (int64_t)s->arena.largest()};
    for (int i = 0; i < ncounters && i < (int)(sizeof v / sizeof v[0]); ++i) counters[i] = v[i];
    return NLS_OK;
}

int nls_server_destroy(nls_server_t s)
{
    if (!s) return NLS_E_INVALID;
    s->stop = true;
    s->cv_work.notify_all();
    if (s->thr.joinable()) s->thr.join();
    for (auto h : s->workers) nls_batch_destroy(h);
    for (auto st : s->streams) cudaStreamDestroy(st);
    if (s->arena_d) cudaFree(s->arena_d);
    delete s;
    return NLS_OK;
}

} // extern "C"
