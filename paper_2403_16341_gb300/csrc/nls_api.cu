// nls_api.cu -- the C ABI (include/nls.h): handles, argument checks, request
// grouping, launches, completion.  Every solve step runs in the kernels; this
// file only validates, allocates library workspace and enqueues.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/nls.h"
#include "nls_internal.h"

// (no `using namespace nls`: its exp overloads must not leak into global lookup)
using nls::KernelInfo;
using nls::SolveArgs;
using nls::FAM_CUBIC;
using nls::FAM_BRATU;
using nls::FAM_SQUARE;
using nls::FAM_ROSENBROCK;
using nls::thread_kernel;
using nls::warp_kernel;
using nls::cta_kernel;

namespace {

constexpr int RING = 1 << 16; // per-handle device counters (2 per request)

struct Request {
    int64_t id = 0;
    SolveArgs args{};
    KernelInfo kern{};
    int family = 0, tiles = 0, lanes = 0, refill = -1;
    int alg_flags = 0;             // the alg word as submitted (precision and tiling flags)
    bool poly = false;             // NLS_POLYALG: the stages of launch_poly
    void *poly_ws = nullptr;       // its device workspace (freed at completion)
    size_t poly_bytes = 0;
    double rate = 0.0;                     // tuned rate (0 = use the cost model)
    int slot = -1;                         // first of 2 ring entries (solved, work counter)
    std::shared_ptr<cudaEvent_t> done;     // recorded after the request's group
    bool launched = false;
    long long solved_final = -1;           // captured when the ring slot is reused
};

struct Opts {
    int persistent = 1;     // persistent grid with a work counter
    int refill_below = 24;  // refill idle lanes when running lanes <= this
    int ctas_per_sm = 0;    // 0 = occupancy limit
    int graph = 1;          // flush through a cached CUDA graph
    int64_t deadline_us = 0; // per-launch iteration budget (0 = none)
};

// Autotuner result for one (family, n, algorithm, precision).
struct Tuned {
    int tiles = 0;      // NLS_TILE_THREAD / WARP / CTA
    int lanes = 0;      // warp tiling: lanes per instance
    int refill = -1;    // REFILL_STATIC: one-block-per-chunk grid; -1: persistent with the
                        // handle's refill threshold; >= 0: persistent with this threshold
    double rate = 0.0;  // measured instances per second on the whole GPU
};
constexpr int REFILL_STATIC = -2;

// A request on host buffers (nls_solve_host_async): its chunk requests, its
// staging block, and its events (the last one follows its copies back).
struct HostReq {
    std::vector<int64_t> chunks;
    void *stage = nullptr;
    size_t stage_bytes = 0;
    std::vector<cudaEvent_t> evs;
    cudaEvent_t done = nullptr;
};

inline long long tune_key(int family, int n, int alg)
{
    return ((long long)family << 40) | ((long long)n << 24) | (long long)(alg & (NLS_ALG_MASK | NLS_MIXED));
}

} // namespace

struct nls_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    size_t mem_cap = 0;
    size_t mem_used = 0;
    int sms = 0;
    std::string err;
    int64_t next_id = 1;
    int64_t launches = 0;
    Opts opt;
    std::map<int64_t, Request> reqs;
    std::vector<int64_t> pending;
    unsigned long long *d_ctr = nullptr; // [RING]
    unsigned long long *h_ctr = nullptr; // pinned mirror
    std::vector<int64_t> owner;          // ring slot -> request id (0 = free)
    int ring_pos = 0;
    // nls_solve_host / nls_solve_host_async: staging blocks not in use (by
    // size), events not in use, and the requests in flight
    std::multimap<size_t, void *> stage_free;
    std::vector<cudaEvent_t> ev_free;
    std::map<int64_t, HostReq> hreqs;
    // cached executable graphs by request-shape signature
    std::map<std::string, cudaGraphExec_t> graphs;
    std::map<const void *, int> occ_cache;
    std::map<long long, Tuned> tuned;
    double *d_tune = nullptr; // autotuner scratch for a prefix of u
    size_t tune_bytes = 0;
    // the host entry points' copy streams and second solve stream (created on
    // first use), and the stream flushes launch on while a host request's
    // chunks alternate between the handle's stream and s_alt (null: the
    // handle's stream)
    cudaStream_t s_in = nullptr, s_out = nullptr, s_alt = nullptr;
    cudaStream_t ls = nullptr;
};

static cudaStream_t launch_stream(const nls_batch *h) { return h->ls ? h->ls : h->stream; }

static std::mutex g_err_mu;
static std::string g_err;

static int fail(nls_batch *h, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    else {
        std::lock_guard<std::mutex> g(g_err_mu);
        g_err = buf;
    }
    return code;
}

int nls::set_global_error(int code, const char *msg) { return fail(nullptr, code, "%s", msg); }

#define NLS_CUDA(h, call)                                                                      \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail((h), NLS_E_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));      \
    } while (0)

static int n_params(int family, int n)
{
    switch (family) {
    case FAM_CUBIC: return n * n + n;
    case FAM_BRATU: return 1;
    case FAM_SQUARE: return n;
    case FAM_ROSENBROCK: return 0;
    default: return -1;
    }
}

static int dev_alloc(nls_batch *h, void **p, size_t bytes)
{
    if (h->mem_cap && h->mem_used + bytes > h->mem_cap)
        return fail(h, NLS_E_NOMEM, "workspace of %zu bytes exceeds the cap of %zu", h->mem_used + bytes,
                    h->mem_cap);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(h, NLS_E_NOMEM, "cudaMalloc(%zu) out of memory", bytes);
    }
    if (e != cudaSuccess) return fail(h, NLS_E_CUDA, "cudaMalloc: %s", cudaGetErrorString(e));
    h->mem_used += bytes;
    return NLS_OK;
}

// Pick the kernel for one request: a forced tiling flag, else the autotuned
// choice for (family, n, algorithm, precision), else thread (n <= 8), warp
// (n <= 32) or CTA (n <= 128).
static int select_kernel(nls_batch *h, int family, int n, int alg, KernelInfo *out, int *tiles_out,
                         int *lanes_out, int *refill_out, double *rate_out)
{
    const bool mixed = (alg & NLS_MIXED) != 0;
    const bool analytic = (alg & NLS_ANALYTIC_JAC) != 0;
    int tiles = alg & (NLS_TILE_THREAD | NLS_TILE_WARP | NLS_TILE_CTA);
    int lanes = 0, refill = -1;
    double rate = 0.0;
    if (tiles && (tiles & (tiles - 1)))
        return fail(h, NLS_E_INVALID, "more than one tiling flag in alg 0x%x", alg);
    if (!tiles) {
        auto it = h->tuned.find(tune_key(family, n, alg));
        if (it != h->tuned.end()) {
            tiles = it->second.tiles;
            lanes = it->second.lanes;
            refill = it->second.refill;
            rate = it->second.rate;
        }
    }
    if ((alg & NLS_ALG_MASK) >= NLS_POTRA_PTAK) {
        const int a = alg & NLS_ALG_MASK;
        if (analytic) return fail(h, NLS_E_UNSUPPORTED, "algorithm %d takes derivatives by forward mode only", a);
        if (!tiles) tiles = n <= 8 ? NLS_TILE_THREAD : n <= 32 ? NLS_TILE_WARP : NLS_TILE_CTA;
        if (tiles == NLS_TILE_THREAD) {
            if (n > 8) return fail(h, NLS_E_UNSUPPORTED, "thread tiling holds n <= 8 (n = %d)", n);
            *out = nls::thread_ext_kernel(family, n, a, mixed);
        } else if (tiles == NLS_TILE_WARP) {
            if (n > 32) return fail(h, NLS_E_UNSUPPORTED, "warp tiling holds n <= 32 (n = %d)", n);
            int L = (lanes == 16 || lanes == 32) && lanes >= n ? lanes : (n <= 16 ? 16 : 32);
            lanes = L;
            *out = nls::warp_ext_kernel(family, L, a, mixed);
        } else {
            *out = nls::cta_ext_kernel(family, n, a, mixed);
        }
    } else if (alg & NLS_REFINE) {
        tiles = NLS_TILE_CTA; // the refined solve is built on the CTA tiling only
    } else {
        if (!tiles) tiles = n <= 8 ? NLS_TILE_THREAD : n <= 32 ? NLS_TILE_WARP : NLS_TILE_CTA;
    }
    if ((alg & NLS_ALG_MASK) >= NLS_POTRA_PTAK) {
        // kernel chosen above
    } else if (tiles == NLS_TILE_THREAD) {
        if (n > 8) return fail(h, NLS_E_UNSUPPORTED, "thread tiling holds n <= 8 (n = %d)", n);
        *out = thread_kernel(family, n, mixed, analytic);
    } else if (tiles == NLS_TILE_WARP) {
        if (n > 32) return fail(h, NLS_E_UNSUPPORTED, "warp tiling holds n <= 32 (n = %d)", n);
        *out = warp_kernel(family, n, mixed, lanes);
    } else {
        *out = cta_kernel(family, n, mixed);
    }
    if (!out->launch) return fail(h, NLS_E_UNSUPPORTED, "no kernel for family %d, n = %d", family, n);
    if (tiles_out) *tiles_out = tiles;
    if (lanes_out) *lanes_out = lanes;
    if (refill_out) *refill_out = refill;
    if (rate_out) *rate_out = rate;
    return NLS_OK;
}

static int occupancy(nls_batch *h, const KernelInfo &k, int *occ)
{
    auto it = h->occ_cache.find(k.func);
    if (it != h->occ_cache.end()) {
        *occ = it->second;
        return NLS_OK;
    }
    int o = 0;
    NLS_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k.func, k.block, k.smem));
    h->occ_cache[k.func] = o;
    *occ = o;
    return NLS_OK;
}

static int wait_event(nls_batch *h, cudaEvent_t ev, int timeout_ms)
{
    if (timeout_ms < 0) {
        NLS_CUDA(h, cudaEventSynchronize(ev));
        return NLS_OK;
    }
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return NLS_OK;
        if (e != cudaErrorNotReady) return fail(h, NLS_E_CUDA, "cudaEventQuery: %s", cudaGetErrorString(e));
        auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0)
                      .count();
        if (ms >= timeout_ms) return fail(h, NLS_E_TIMEOUT, "request not complete after %d ms", timeout_ms);
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

// Reserve `count` consecutive ring entries; requests still owning them are
// waited for and their solved counts kept on the host first.
static int ring_take(nls_batch *h, int count, int *start)
{
    if (count > RING) return fail(h, NLS_E_INVALID, "too many requests in one flush (%d)", count / 2);
    if (h->ring_pos + count > RING) h->ring_pos = 0;
    const int s = h->ring_pos;
    for (int i = s; i < s + count; ++i) {
        const int64_t id = h->owner[i];
        if (!id) continue;
        auto it = h->reqs.find(id);
        if (it != h->reqs.end() && it->second.slot >= 0) {
            Request &r = it->second;
            NLS_CUDA(h, cudaEventSynchronize(*r.done));
            r.solved_final = (long long)h->h_ctr[r.slot];
            h->owner[r.slot] = h->owner[r.slot + 1] = 0;
            r.slot = -1;
        }
        h->owner[i] = 0;
    }
    h->ring_pos = s + count;
    *start = s;
    return NLS_OK;
}

// Launch geometry of every pending request.  A lone request runs as a
// persistent grid (one wave of CTAs drawing instances from its work counter,
// lanes refilled as instances finish).  When several requests are flushed
// together (the buckets of an uneven batch, a serving wave), every kernel
// gets its full one-block-per-chunk grid instead: the hardware interleaves
// the CTAs of the concurrent graph nodes as they retire, which keeps the
// GPU full without any cost model (a fixed split into small persistent
// grids leaves SMs idle when only a few kernels run concurrently).
static int plan_grids(nls_batch *h, const std::vector<Request *> &rs, std::vector<int> &grids)
{
    int live = 0;
    for (Request *r : rs)
        if (r->args.batch > 0 && !r->poly) ++live;
    grids.assign(rs.size(), 0);
    for (size_t i = 0; i < rs.size(); ++i) {
        Request &r = *rs[i];
        if (r.args.batch == 0 || r.poly) continue; // a poly request runs its own chain
        const int64_t ctas = (r.args.batch + r.kern.per_cta - 1) / r.kern.per_cta;
        const bool persistent = h->opt.persistent && live == 1 && r.refill != REFILL_STATIC;
        if (!persistent) {
            grids[i] = (int)std::min<int64_t>(ctas, INT32_MAX);
            r.args.counter = nullptr;
            r.args.refill_below = 0;
            continue;
        }
        int occ = 0;
        int rc = occupancy(h, r.kern, &occ);
        if (rc) return rc;
        if (h->opt.ctas_per_sm > 0) occ = std::min(occ, h->opt.ctas_per_sm);
        grids[i] = (int)std::min<int64_t>(ctas, (int64_t)std::max(occ, 1) * h->sms);
        r.args.counter = h->d_ctr + r.slot + 1;
        r.args.refill_below = r.refill >= 0 ? r.refill : h->opt.refill_below;
    }
    return NLS_OK;
}

// Memset of the group's counters -> one kernel node per request (no edges
// between them, so they run concurrently) -> copy of the counters to the
// host.  The executable graph is cached by the shape of the group and
// updated in place on later flushes of the same shape.
static int launch_graph(nls_batch *h, const std::vector<Request *> &rs, const std::vector<int> &grids, int s0,
                        int nctr)
{
    std::ostringstream sig;
    cudaGraph_t g = nullptr;
    NLS_CUDA(h, cudaGraphCreate(&g, 0));
    struct Guard {
        cudaGraph_t g;
        ~Guard() { cudaGraphDestroy(g); }
    } guard{g};
    cudaMemsetParams mp{};
    mp.dst = h->d_ctr + s0;
    mp.value = 0;
    mp.elementSize = 4;
    mp.width = (size_t)nctr * 2;
    mp.height = 1;
    cudaGraphNode_t ms = nullptr;
    NLS_CUDA(h, cudaGraphAddMemsetNode(&ms, g, nullptr, 0, &mp));
    std::vector<cudaGraphNode_t> kn;
    int64_t launched = 0;
    for (size_t i = 0; i < rs.size(); ++i) {
        if (!grids[i]) continue;
        Request &r = *rs[i];
        void *kargs[] = {&r.args};
        cudaKernelNodeParams kp{};
        kp.func = const_cast<void *>(r.kern.func);
        kp.gridDim = dim3(grids[i]);
        kp.blockDim = dim3(r.kern.block);
        kp.sharedMemBytes = r.kern.smem;
        kp.kernelParams = kargs;
        cudaGraphNode_t node = nullptr;
        NLS_CUDA(h, cudaGraphAddKernelNode(&node, g, &ms, 1, &kp));
        kn.push_back(node);
        ++launched;
    }
    cudaGraphNode_t cp = nullptr;
    NLS_CUDA(h, cudaGraphAddMemcpyNode1D(&cp, g, kn.empty() ? &ms : kn.data(), kn.empty() ? 1 : kn.size(),
                                         h->h_ctr + s0, h->d_ctr + s0, sizeof(unsigned long long) * nctr,
                                         cudaMemcpyDeviceToHost));
    // The cache key is the graph's shape only: cudaGraphExecUpdate takes a
    // kernel node's new function, grid and arguments, so every flush with the
    // same number of kernels reuses one executable graph.  (Keyed by the
    // kernel list, a server's waves of mixed requests would instantiate a new
    // graph for most waves, at a few hundred microseconds each.)
    sig << launched << '#' << nctr << '@' << (const void *)launch_stream(h);
    const std::string key = sig.str();
    auto it = h->graphs.find(key);
    cudaGraphExec_t exec = nullptr;
    if (it != h->graphs.end()) {
        cudaGraphExecUpdateResultInfo info{};
        if (cudaGraphExecUpdate(it->second, g, &info) == cudaSuccess) {
            exec = it->second;
        } else {
            cudaGetLastError();
            cudaGraphExecDestroy(it->second);
            h->graphs.erase(it);
        }
    }
    if (!exec) {
        if (h->graphs.size() >= 64) {
            cudaGraphExecDestroy(h->graphs.begin()->second);
            h->graphs.erase(h->graphs.begin());
        }
        NLS_CUDA(h, cudaGraphInstantiate(&exec, g, 0));
        h->graphs[key] = exec;
    }
    NLS_CUDA(h, cudaGraphLaunch(exec, launch_stream(h)));
    h->launches += launched;
    return NLS_OK;
}

static int launch_direct(nls_batch *h, const std::vector<Request *> &rs, const std::vector<int> &grids, int s0,
                         int nctr)
{
    const cudaStream_t st = launch_stream(h);
    NLS_CUDA(h, cudaMemsetAsync(h->d_ctr + s0, 0, sizeof(unsigned long long) * nctr, st));
    for (size_t i = 0; i < rs.size(); ++i) {
        if (!grids[i]) continue;
        cudaError_t e = rs[i]->kern.launch(rs[i]->args, grids[i], st);
        if (e != cudaSuccess) return fail(h, NLS_E_CUDA, "kernel launch: %s", cudaGetErrorString(e));
        ++h->launches;
    }
    NLS_CUDA(h, cudaMemcpyAsync(h->h_ctr + s0, h->d_ctr + s0, sizeof(unsigned long long) * nctr,
                                cudaMemcpyDeviceToHost, st));
    return NLS_OK;
}

// Device workspace of a poly-algorithm request: the original u0, compact
// copies of the instances still failing, their outputs, full-size outputs the
// caller did not provide, and the stage counters.
// Stages of the poly-algorithm (Sec. 3.2, Fig. 4): a quasi-Newton phase
// (Broyden, then modified Broyden; Klement is not built) for n > 25, then
// Newton, backtracking, trust region.  For n <= 25 the quasi-Newton phase
// is skipped, as in the paper.
constexpr int POLY_MAX_STAGES = 5;
constexpr int POLY_QN_MIN_N = 26;

struct PolyWs {
    double *u0, *cparams, *cu, *cres, *fres;
    int64_t *idx;
    int32_t *cst, *cit, *cnf, *fst, *fit, *fnf;
    unsigned long long *ctr; // per gathered stage s: [3s] gathered, [3s+1] solved, [3s+2] work
};

static size_t poly_layout(int64_t B, int n, int E, char *base, PolyWs *w)
{
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off += al(bytes);
        return p;
    };
    PolyWs t{};
    t.u0 = (double *)take((size_t)n * B * 8);
    t.cparams = (double *)take((size_t)std::max(E, 1) * B * 8);
    t.cu = (double *)take((size_t)n * B * 8);
    t.cres = (double *)take((size_t)B * 8);
    t.fres = (double *)take((size_t)B * 8);
    t.idx = (int64_t *)take((size_t)B * 8);
    t.cst = (int32_t *)take((size_t)B * 4);
    t.cit = (int32_t *)take((size_t)B * 4);
    t.cnf = (int32_t *)take((size_t)B * 4);
    t.fst = (int32_t *)take((size_t)B * 4);
    t.fit = (int32_t *)take((size_t)B * 4);
    t.fnf = (int32_t *)take((size_t)B * 4);
    t.ctr = (unsigned long long *)take(POLY_MAX_STAGES * 3 * 8);
    if (w) *w = t;
    return off;
}

// Newton on every instance; the failures restart from u0 with backtracking;
// what still fails restarts with the trust region (Sec. 3.2).  All on the
// handle's stream, counts kept on the device.
static int launch_poly(nls_batch *h, Request &r)
{
    const int64_t B = r.args.batch;
    const int n = r.args.n, E = n_params(r.family, n);
    const bool mixed = (r.alg_flags & NLS_MIXED) != 0;
    PolyWs w;
    poly_layout(B, n, E, static_cast<char *>(r.poly_ws), &w);
    cudaStream_t st = launch_stream(h);
    SolveArgs a = r.args;
    if (!a.status) a.status = w.fst;
    if (!a.iters) a.iters = w.fit;
    if (!a.nfev) a.nfev = w.fnf;
    if (!a.resid) a.resid = w.fres;
    // the stages' gradient counts are not kept: ngrad reads 0 for a poly request
    if (a.ngrad) NLS_CUDA(h, cudaMemsetAsync(a.ngrad, 0, (size_t)B * 4, st));
    a.ngrad = nullptr;
    NLS_CUDA(h, cudaMemcpyAsync(w.u0, a.u, (size_t)n * B * 8, cudaMemcpyDeviceToDevice, st));
    NLS_CUDA(h, cudaMemsetAsync(w.ctr, 0, POLY_MAX_STAGES * 3 * 8, st));
    int stages[POLY_MAX_STAGES], ns = 0;
    if (n >= POLY_QN_MIN_N) {
        stages[ns++] = NLS_BROYDEN;
        stages[ns++] = NLS_MOD_BROYDEN;
    }
    stages[ns++] = NLS_NEWTON;
    stages[ns++] = NLS_NEWTON_BACKTRACK;
    stages[ns++] = NLS_TRUST_DOGLEG;
    // the kernel of a stage: the request's tiling; Broyden's on the same tiling
    auto stage_kernel = [&](int alg) -> KernelInfo {
        if (alg < NLS_BROYDEN) return r.kern;
        if (r.tiles == NLS_TILE_WARP) return nls::warp_ext_kernel(r.family, n <= 16 ? 16 : 32, alg, mixed);
        return nls::cta_ext_kernel(r.family, n, alg, mixed);
    };
    // first stage on the whole batch
    KernelInfo k0 = stage_kernel(stages[0]);
    if (!k0.launch) return fail(h, NLS_E_UNSUPPORTED, "no poly stage kernel for family %d, n = %d", r.family, n);
    a.alg = stages[0];
    a.counter = nullptr;
    a.refill_below = 0;
    const int64_t ctas0 = (B + k0.per_cta - 1) / k0.per_cta;
    cudaError_t e = k0.launch(a, (int)std::min<int64_t>(ctas0, INT32_MAX), st);
    if (e != cudaSuccess) return fail(h, NLS_E_CUDA, "poly stage 1: %s", cudaGetErrorString(e));
    ++h->launches;
    for (int sidx = 1; sidx < ns; ++sidx) {
        const KernelInfo ks = stage_kernel(stages[sidx]);
        if (!ks.launch) return fail(h, NLS_E_UNSUPPORTED, "no poly stage kernel for family %d, n = %d", r.family, n);
        int occ = 0;
        int rc = occupancy(h, ks, &occ);
        if (rc) return rc;
        const int64_t ctas = (B + ks.per_cta - 1) / ks.per_cta;
        const int grid = (int)std::min<int64_t>(ctas, (int64_t)std::max(occ, 1) * h->sms);
        unsigned long long *cnt = w.ctr + 3 * (sidx - 1);
        nls::PolyGatherArgs g{B, E, n, a.status, a.params, w.u0, w.idx, w.cparams, w.cu, cnt};
        e = nls::launch_poly_gather(g, st);
        if (e != cudaSuccess) return fail(h, NLS_E_CUDA, "poly gather: %s", cudaGetErrorString(e));
        SolveArgs c = a;
        c.params = E ? w.cparams : nullptr;
        c.u = w.cu;
        c.batch = B;
        c.ld = B;
        c.dyn_batch = cnt;
        c.alg = stages[sidx];
        c.status = w.cst;
        c.iters = w.cit;
        c.nfev = w.cnf;
        c.resid = w.cres;
        c.solved = cnt + 1;
        c.counter = cnt + 2;
        c.refill_below = h->opt.refill_below;
        e = ks.launch(c, grid, st);
        if (e != cudaSuccess) return fail(h, NLS_E_CUDA, "poly stage %d: %s", sidx + 1, cudaGetErrorString(e));
        nls::PolyScatterArgs sc{B, n, cnt, w.idx, w.cu, w.cst, w.cit, w.cnf, w.cres,
                                a.u, a.status, a.iters, a.nfev, a.resid};
        e = nls::launch_poly_scatter(sc, st);
        if (e != cudaSuccess) return fail(h, NLS_E_CUDA, "poly scatter: %s", cudaGetErrorString(e));
        h->launches += 3;
    }
    e = nls::launch_poly_total(a.solved, w.ctr, ns - 1, st);
    if (e != cudaSuccess) return fail(h, NLS_E_CUDA, "poly total: %s", cudaGetErrorString(e));
    ++h->launches;
    return NLS_OK;
}

static int flush_pending(nls_batch *h)
{
    if (h->pending.empty()) return NLS_OK;
    const int nreq = (int)h->pending.size();
    int s0 = 0;
    int rc = ring_take(h, 2 * nreq, &s0);
    if (rc) return rc;
    auto ev = std::shared_ptr<cudaEvent_t>(new cudaEvent_t, [](cudaEvent_t *e) {
        cudaEventDestroy(*e);
        delete e;
    });
    NLS_CUDA(h, cudaEventCreateWithFlags(ev.get(), cudaEventDisableTiming));
    std::vector<Request *> rs;
    for (int i = 0; i < nreq; ++i) {
        Request &r = h->reqs[h->pending[i]];
        r.slot = s0 + 2 * i;
        h->owner[r.slot] = h->owner[r.slot + 1] = r.id;
        r.args.solved = h->d_ctr + r.slot;
        r.done = ev;
        r.launched = true;
        rs.push_back(&r);
    }
    std::vector<int> grids;
    rc = plan_grids(h, rs, grids);
    if (rc) return rc;
    rc = h->opt.graph ? launch_graph(h, rs, grids, s0, 2 * nreq) : launch_direct(h, rs, grids, s0, 2 * nreq);
    if (rc) return rc;
    bool any_poly = false;
    for (Request *r : rs)
        if (r->poly && r->args.batch > 0) {
            rc = launch_poly(h, *r);
            if (rc) return rc;
            any_poly = true;
        }
    if (any_poly)
        NLS_CUDA(h, cudaMemcpyAsync(h->h_ctr + s0, h->d_ctr + s0, sizeof(unsigned long long) * 2 * nreq,
                                    cudaMemcpyDeviceToHost, launch_stream(h)));
    NLS_CUDA(h, cudaEventRecord(*ev, launch_stream(h)));
    h->pending.clear();
    return NLS_OK;
}

static int validate(nls_batch *h, int family, const double *params, const double *u, int n, int64_t batch,
                    int alg, double abstol, int maxiters)
{
    if (!h) return NLS_E_INVALID;
    if (family < 0 || family > FAM_ROSENBROCK) return fail(h, NLS_E_UNSUPPORTED, "unknown family %d", family);
    if (n < 1 || n > 128) return fail(h, NLS_E_UNSUPPORTED, "n = %d outside [1, 128]", n);
    if (batch < 0) return fail(h, NLS_E_INVALID, "negative batch");
    if (maxiters < 0) return fail(h, NLS_E_INVALID, "negative maxiters");
    if (!(abstol >= 0.0) || !std::isfinite(abstol)) return fail(h, NLS_E_INVALID, "abstol must be finite and >= 0");
    const int a = alg & NLS_ALG_MASK;
    if (a > NLS_MOD_BROYDEN) return fail(h, NLS_E_INVALID, "unknown algorithm %d", a);
    if (alg & ~(NLS_ALG_MASK | NLS_MIXED | NLS_ANALYTIC_JAC | NLS_TILE_THREAD | NLS_TILE_WARP | NLS_TILE_CTA |
                NLS_TR_NOCEDAL_WRIGHT | NLS_REFINE))
        return fail(h, NLS_E_INVALID, "unknown flags in alg 0x%x", alg);
    if ((alg & NLS_REFINE) && (!(alg & NLS_MIXED) || a > NLS_TRUST_DOGLEG || (alg & (NLS_TILE_THREAD | NLS_TILE_WARP))))
        return fail(h, NLS_E_UNSUPPORTED,
                    "NLS_REFINE refines the FP32 solves of NLS_MIXED Newton, backtracking or trust region on the "
                    "CTA tiling (alg 0x%x)", alg);
    if ((alg & NLS_TR_NOCEDAL_WRIGHT) && a != NLS_TRUST_DOGLEG && a != NLS_POLYALG)
        return fail(h, NLS_E_INVALID, "NLS_TR_NOCEDAL_WRIGHT needs a trust-region algorithm (alg %d)", a);
    if (batch > 0 && !u) return fail(h, NLS_E_INVALID, "u is NULL");
    if (batch > 0 && n_params(family, n) > 0 && !params) return fail(h, NLS_E_INVALID, "params is NULL");
    return NLS_OK;
}

static int load_tuning(nls_batch *h, const char *path)
{
    std::ifstream f(path);
    if (!f) return fail(h, NLS_E_INVALID, "cannot read tuning table %s", path);
    std::string line;
    int loaded = 0;
    while (std::getline(f, line)) {
        if (line.empty() || line[0] == '#') continue;
        std::istringstream is(line);
        int fam, n, alg;
        Tuned t;
        if (is >> fam >> n >> alg >> t.tiles >> t.lanes >> t.refill >> t.rate) {
            h->tuned[tune_key(fam, n, alg)] = t;
            ++loaded;
        }
    }
    return loaded;
}

// One timed trial of a tiling on the first S instances of a request; u's
// prefix is restored from `save` before the run.
static int tune_trial(nls_batch *h, const SolveArgs &base, const KernelInfo &k, int refill, const double *save,
                      int64_t save_pitch, int64_t S, unsigned long long *ctr, float *ms_out)
{
    SolveArgs a = base;
    a.batch = S;
    a.solved = ctr;
    a.counter = refill == REFILL_STATIC ? nullptr : ctr + 1;
    a.refill_below = refill >= 0 ? refill : refill == REFILL_STATIC ? 0 : h->opt.refill_below;
    a.status = nullptr;
    a.iters = nullptr;
    a.resid = nullptr;
    a.nfev = nullptr;
    a.ngrad = nullptr;
    int occ = 0;
    int rc = occupancy(h, k, &occ);
    if (rc) return rc;
    const int64_t ctas = (S + k.per_cta - 1) / k.per_cta;
    const int grid = refill == REFILL_STATIC ? (int)std::min<int64_t>(ctas, INT32_MAX)
                                             : (int)std::min<int64_t>(ctas, (int64_t)std::max(occ, 1) * h->sms);
    cudaEvent_t e0, e1;
    NLS_CUDA(h, cudaEventCreate(&e0));
    NLS_CUDA(h, cudaEventCreate(&e1));
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        NLS_CUDA(h, cudaMemcpy2DAsync(base.u, base.ld * 8, save, save_pitch * 8, S * 8, base.n,
                                      cudaMemcpyDeviceToDevice, h->stream));
        NLS_CUDA(h, cudaMemsetAsync(ctr, 0, 16, h->stream));
        NLS_CUDA(h, cudaEventRecord(e0, h->stream));
        cudaError_t e = k.launch(a, grid, h->stream);
        if (e != cudaSuccess) return fail(h, NLS_E_CUDA, "tuning launch: %s", cudaGetErrorString(e));
        ++h->launches;
        NLS_CUDA(h, cudaEventRecord(e1, h->stream));
        NLS_CUDA(h, cudaEventSynchronize(e1));
        float ms = 0.f;
        NLS_CUDA(h, cudaEventElapsedTime(&ms, e0, e1));
        best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_out = best;
    return NLS_OK;
}

extern "C" {

int nls_batch_create(nls_handle *out, int device, void *cuda_stream, size_t mem_cap_bytes)
{
    if (!out) return fail(nullptr, NLS_E_INVALID, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return fail(nullptr, NLS_E_CUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
    if (device < 0 || device >= ndev) return fail(nullptr, NLS_E_INVALID, "device %d of %d", device, ndev);
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail(nullptr, NLS_E_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    std::unique_ptr<nls_batch> h(new nls_batch);
    h->device = device;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->mem_cap = mem_cap_bytes;
    cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, device);
    int rc = dev_alloc(h.get(), (void **)&h->d_ctr, sizeof(unsigned long long) * RING);
    if (rc) return fail(nullptr, rc, "%s", h->err.c_str());
    e = cudaMallocHost((void **)&h->h_ctr, sizeof(unsigned long long) * RING);
    if (e != cudaSuccess) {
        cudaFree(h->d_ctr);
        return fail(nullptr, NLS_E_CUDA, "cudaMallocHost: %s", cudaGetErrorString(e));
    }
    h->owner.assign(RING, 0);
    if (const char *cache = std::getenv("NLS_TUNE_CACHE")) load_tuning(h.get(), cache);
    *out = h.release();
    return NLS_OK;
}

// Enqueue one request on instances [0, batch) of arrays with leading
// dimension ld >= batch (element e of instance k at [e * ld + k]).
static int enqueue(nls_batch *h, int family, const double *params, double *u, int n, int64_t batch, int64_t ld,
                   int alg, double abstol, int maxiters, const nls_outputs *out, int64_t *req)
{
    int rc = 0;
    Request r;
    rc = select_kernel(h, family, n, alg, &r.kern, &r.tiles, &r.lanes, &r.refill, &r.rate);
    if (rc) return rc;
    r.family = family;
    r.id = h->next_id++;
    r.args.params = params;
    r.args.u = u;
    r.args.batch = batch;
    r.args.ld = ld;
    r.args.n = n;
    r.args.alg = alg & NLS_ALG_MASK;
    r.alg_flags = alg;
    r.args.tr_scheme = (alg & NLS_TR_NOCEDAL_WRIGHT) ? nls::TR_NOCEDAL_WRIGHT : nls::TR_SIMPLE;
    r.args.refine = (alg & NLS_REFINE) ? 2 : 0;
    r.args.abstol = abstol;
    r.args.maxiters = maxiters;
    r.args.budget_ns = (unsigned long long)h->opt.deadline_us * 1000ull;
    if (out) {
        r.args.status = out->status;
        r.args.iters = out->iters;
        r.args.resid = out->resid_inf;
        r.args.nfev = out->nfev;
        r.args.ngrad = out->ngrad;
    }
    if ((alg & NLS_ALG_MASK) == NLS_POLYALG) {
        r.poly = true;
        if (batch > 0) {
            r.poly_bytes = poly_layout(batch, n, n_params(family, n), nullptr, nullptr);
            rc = dev_alloc(h, &r.poly_ws, r.poly_bytes);
            if (rc) return rc;
        }
    }
    h->reqs[r.id] = r;
    h->pending.push_back(r.id);
    *req = r.id;
    return NLS_OK;
}

int nls_solve(nls_handle h, int family, const double *params, double *u, int n, int64_t batch, int alg,
              double abstol, int maxiters, const nls_outputs *out, int64_t *req)
{
    int rc = validate(h, family, params, u, n, batch, alg, abstol, maxiters);
    if (rc) return rc;
    if (!req) return fail(h, NLS_E_INVALID, "req is NULL");
    return enqueue(h, family, params, u, n, batch, batch, alg, abstol, maxiters, out, req);
}

int nls_flush(nls_handle h)
{
    if (!h) return NLS_E_INVALID;
    NLS_CUDA(h, cudaSetDevice(h->device));
    return flush_pending(h);
}

static int host_status(nls_handle h, int64_t req, int64_t *solved, int timeout_ms);

int nls_status(nls_handle h, int64_t req, int64_t *solved, int timeout_ms)
{
    if (!h) return NLS_E_INVALID;
    if (h->hreqs.count(req)) return host_status(h, req, solved, timeout_ms);
    auto it = h->reqs.find(req);
    if (it == h->reqs.end()) return fail(h, NLS_E_NOTFOUND, "unknown request %lld", (long long)req);
    NLS_CUDA(h, cudaSetDevice(h->device));
    if (!it->second.launched) {
        int rc = flush_pending(h);
        if (rc) return rc;
    }
    Request &r = it->second;
    int rc = wait_event(h, *r.done, timeout_ms);
    if (rc) return rc;
    long long s = r.solved_final;
    if (r.slot >= 0) {
        s = (long long)h->h_ctr[r.slot];
        h->owner[r.slot] = h->owner[r.slot + 1] = 0;
    }
    if (solved) *solved = s;
    if (r.poly_ws) {
        cudaFree(r.poly_ws);
        h->mem_used -= r.poly_bytes;
    }
    h->reqs.erase(it);
    return NLS_OK;
}

// Staging block of at least `need` bytes: the smallest idle block that is
// not more than twice as large, else a new one (idle blocks are released
// first when the memory cap would be exceeded).
static int take_stage(nls_batch *h, size_t need, void **p, size_t *bytes)
{
    auto it = h->stage_free.lower_bound(need);
    if (it != h->stage_free.end() && it->first <= 2 * need) {
        *p = it->second;
        *bytes = it->first;
        h->stage_free.erase(it);
        return NLS_OK;
    }
    if (h->mem_cap && h->mem_used + need > h->mem_cap) {
        for (auto &kv : h->stage_free) {
            cudaFree(kv.second);
            h->mem_used -= kv.first;
        }
        h->stage_free.clear();
    }
    int rc = dev_alloc(h, p, need);
    if (rc) return rc;
    *bytes = need;
    return NLS_OK;
}

static int take_event(nls_batch *h, cudaEvent_t *e)
{
    if (!h->ev_free.empty()) {
        *e = h->ev_free.back();
        h->ev_free.pop_back();
        return NLS_OK;
    }
    NLS_CUDA(h, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    return NLS_OK;
}

// Completion of a host request: its copies back are done (which follow every
// chunk's solve), then the chunks' solved counts; the staging block and the
// events go back to the handle's pools.
static int host_status(nls_handle h, int64_t req, int64_t *solved, int timeout_ms)
{
    NLS_CUDA(h, cudaSetDevice(h->device));
    HostReq &q = h->hreqs[req];
    int rc = wait_event(h, q.done, timeout_ms);
    if (rc) return rc;
    int64_t total = 0;
    for (int64_t c : q.chunks) {
        int64_t sv = 0;
        rc = nls_status(h, c, &sv, -1);
        if (rc) return rc;
        total += sv;
    }
    h->stage_free.emplace(q.stage_bytes, q.stage);
    for (cudaEvent_t e : q.evs) h->ev_free.push_back(e);
    h->hreqs.erase(req);
    if (solved) *solved = total;
    return NLS_OK;
}

int nls_solve_host_async(nls_handle h, int family, const double *params, double *u, int n, int64_t batch,
                         int alg, double abstol, int maxiters, const nls_outputs *out, int64_t *req)
{
    int rc = validate(h, family, params, u, n, batch, alg, abstol, maxiters);
    if (rc) return rc;
    if (!req) return fail(h, NLS_E_INVALID, "req is NULL");
    NLS_CUDA(h, cudaSetDevice(h->device));
    // requests made with nls_solve before this call launch on the handle's
    // stream, in its order, before any chunk takes the second solve stream
    rc = flush_pending(h);
    if (rc) return rc;
    const size_t E = (size_t)n_params(family, n);
    const size_t bp = E * (size_t)batch * 8, bu = (size_t)n * (size_t)batch * 8, bo = (size_t)batch * 4;
    const size_t need = bp + bu + 4 * bo + (size_t)batch * 8 + 5 * 256;
    HostReq q;
    rc = take_stage(h, need, &q.stage, &q.stage_bytes);
    if (rc) return rc;
    auto align = [](size_t x) { return (x + 255) & ~size_t(255); };
    char *base = static_cast<char *>(q.stage);
    double *dp = reinterpret_cast<double *>(base);
    double *du = reinterpret_cast<double *>(base + align(bp));
    double *dres = reinterpret_cast<double *>(base + align(bp) + align(bu));
    int32_t *dst = reinterpret_cast<int32_t *>(base + align(bp) + align(bu) + align((size_t)batch * 8));
    int32_t *dit = dst + align(bo) / 4;
    int32_t *dnf = dit + align(bo) / 4;
    int32_t *dng = dnf + align(bo) / 4;
    // Large batches are pipelined in chunks of instances: chunk c + 1's inputs
    // go up on s_in while chunk c is solved, and the results of finished
    // chunks come back on s_out; events order the streams.  The chunks' solves
    // alternate between the handle's stream and s_alt, so a chunk's launch can
    // take the SMs its predecessor's persistent grid frees while that grid
    // drains (its tail), instead of every chunk paying its own.  Chunks address
    // the staging arrays with leading dimension `batch`.  The poly-algorithm
    // gathers whole arrays, so it keeps one chunk.  Chunks of at least 2^17
    // instances (several waves of a persistent grid), at most eight.  Requests
    // made one after another queue on the same streams, so a request's
    // uploads overlap the previous request's solves.
    const int64_t C = (alg & NLS_ALG_MASK) == NLS_POLYALG ? 1 : std::min<int64_t>(8, std::max<int64_t>(1, batch >> 17));
    if (C > 1) {
        if (!h->s_in) NLS_CUDA(h, cudaStreamCreateWithFlags(&h->s_in, cudaStreamNonBlocking));
        if (!h->s_out) NLS_CUDA(h, cudaStreamCreateWithFlags(&h->s_out, cudaStreamNonBlocking));
        if (!h->s_alt) NLS_CUDA(h, cudaStreamCreateWithFlags(&h->s_alt, cudaStreamNonBlocking));
    }
    auto give_back = [&]() {
        h->stage_free.emplace(q.stage_bytes, q.stage);
        for (cudaEvent_t e : q.evs) h->ev_free.push_back(e);
    };
    const int nev = C > 1 ? (int)(2 * C) + 1 : 1;
    for (int i = 0; i < nev; ++i) {
        cudaEvent_t e;
        rc = take_event(h, &e);
        if (rc) {
            give_back();
            return rc;
        }
        q.evs.push_back(e);
    }
    q.done = q.evs.back();
    cudaStream_t sin = C > 1 ? h->s_in : h->stream, sout = C > 1 ? h->s_out : h->stream;
#define NLS_HCUDA(call)                                                                                \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) {                                                                       \
            give_back();                                                                               \
            return fail(h, NLS_E_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));              \
        }                                                                                              \
    } while (0)
    for (int64_t c = 0; c < C; ++c) {
        const int64_t k0 = batch * c / C, kc = batch * (c + 1) / C - k0;
        if (bp)
            NLS_HCUDA(cudaMemcpy2DAsync(dp + k0, batch * 8, params + k0, batch * 8, kc * 8, E,
                                        cudaMemcpyHostToDevice, sin));
        if (bu)
            NLS_HCUDA(cudaMemcpy2DAsync(du + k0, batch * 8, u + k0, batch * 8, kc * 8, n, cudaMemcpyHostToDevice,
                                        sin));
        const cudaStream_t ss = (C > 1 && (c & 1)) ? h->s_alt : h->stream; // this chunk's solve
        if (C > 1) {
            NLS_HCUDA(cudaEventRecord(q.evs[2 * c], sin));
            NLS_HCUDA(cudaStreamWaitEvent(ss, q.evs[2 * c], 0));
        }
        nls_outputs dout{out && out->status ? dst + k0 : nullptr, out && out->iters ? dit + k0 : nullptr,
                         out && out->resid_inf ? dres + k0 : nullptr, out && out->nfev ? dnf + k0 : nullptr,
                         out && out->ngrad ? dng + k0 : nullptr};
        int64_t creq = 0;
        rc = enqueue(h, family, bp ? dp + k0 : nullptr, du + k0, n, kc, batch, alg, abstol, maxiters, &dout, &creq);
        if (rc == NLS_OK) {
            h->ls = ss;
            rc = flush_pending(h);
            h->ls = nullptr;
        }
        if (rc) {
            give_back();
            return rc;
        }
        q.chunks.push_back(creq);
        if (C > 1) {
            NLS_HCUDA(cudaEventRecord(q.evs[2 * c + 1], ss));
            NLS_HCUDA(cudaStreamWaitEvent(sout, q.evs[2 * c + 1], 0));
        }
        if (bu)
            NLS_HCUDA(cudaMemcpy2DAsync(u + k0, batch * 8, du + k0, batch * 8, kc * 8, n, cudaMemcpyDeviceToHost,
                                        sout));
        if (out && out->status)
            NLS_HCUDA(cudaMemcpyAsync(out->status + k0, dst + k0, kc * 4, cudaMemcpyDeviceToHost, sout));
        if (out && out->iters)
            NLS_HCUDA(cudaMemcpyAsync(out->iters + k0, dit + k0, kc * 4, cudaMemcpyDeviceToHost, sout));
        if (out && out->nfev)
            NLS_HCUDA(cudaMemcpyAsync(out->nfev + k0, dnf + k0, kc * 4, cudaMemcpyDeviceToHost, sout));
        if (out && out->ngrad)
            NLS_HCUDA(cudaMemcpyAsync(out->ngrad + k0, dng + k0, kc * 4, cudaMemcpyDeviceToHost, sout));
        if (out && out->resid_inf)
            NLS_HCUDA(cudaMemcpyAsync(out->resid_inf + k0, dres + k0, kc * 8, cudaMemcpyDeviceToHost, sout));
    }
    NLS_HCUDA(cudaEventRecord(q.done, sout));
#undef NLS_HCUDA
    const int64_t id = h->next_id++;
    h->hreqs[id] = std::move(q);
    *req = id;
    return NLS_OK;
}

int nls_solve_host(nls_handle h, int family, const double *params, double *u, int n, int64_t batch, int alg,
                   double abstol, int maxiters, const nls_outputs *out, int64_t *solved)
{
    int64_t req = 0;
    int rc = nls_solve_host_async(h, family, params, u, n, batch, alg, abstol, maxiters, out, &req);
    if (rc) return rc;
    return nls_status(h, req, solved, -1);
}

int nls_batch_destroy(nls_handle h)
{
    if (!h) return NLS_E_INVALID;
    cudaSetDevice(h->device);
    flush_pending(h);
    cudaStreamSynchronize(h->stream);
    if (h->s_in) cudaStreamSynchronize(h->s_in);
    if (h->s_out) cudaStreamSynchronize(h->s_out);
    if (h->s_alt) cudaStreamSynchronize(h->s_alt);
    for (auto &kv : h->reqs)
        if (kv.second.poly_ws) cudaFree(kv.second.poly_ws);
    h->reqs.clear();
    for (auto &kv : h->hreqs) {
        if (kv.second.stage) cudaFree(kv.second.stage);
        for (cudaEvent_t e : kv.second.evs) cudaEventDestroy(e);
    }
    h->hreqs.clear();
    for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second);
    if (h->d_tune) cudaFree(h->d_tune);
    for (auto &kv : h->stage_free) cudaFree(kv.second);
    if (h->d_ctr) cudaFree(h->d_ctr);
    if (h->h_ctr) cudaFreeHost(h->h_ctr);
    for (cudaEvent_t e : h->ev_free) cudaEventDestroy(e);
    if (h->s_in) cudaStreamDestroy(h->s_in);
    if (h->s_out) cudaStreamDestroy(h->s_out);
    if (h->s_alt) cudaStreamDestroy(h->s_alt);
    delete h;
    return NLS_OK;
}

const char *nls_last_error(nls_handle h)
{
    if (h) return h->err.c_str();
    std::lock_guard<std::mutex> g(g_err_mu);
    return g_err.c_str();
}

int64_t nls_launch_count(nls_handle h) { return h ? h->launches : 0; }

int nls_autotune(nls_handle h, int family, const double *params, double *u, int n, int64_t batch, int alg,
                 double abstol, int maxiters, int *chosen)
{
    int rc = validate(h, family, params, u, n, batch, alg, abstol, maxiters);
    if (rc) return rc;
    if (alg & (NLS_TILE_THREAD | NLS_TILE_WARP | NLS_TILE_CTA))
        return fail(h, NLS_E_INVALID, "nls_autotune chooses the tiling: pass no tiling flag");
    if (alg & NLS_REFINE) return fail(h, NLS_E_UNSUPPORTED, "NLS_REFINE runs the CTA tiling only: nothing to tune");
    if ((alg & NLS_ALG_MASK) == NLS_POLYALG)
        return fail(h, NLS_E_INVALID, "tune the stage algorithms, not NLS_POLYALG");
    if ((alg & NLS_ALG_MASK) >= NLS_POTRA_PTAK && (alg & NLS_ANALYTIC_JAC))
        return fail(h, NLS_E_UNSUPPORTED, "algorithm %d takes forward-mode derivatives only", alg & NLS_ALG_MASK);
    NLS_CUDA(h, cudaSetDevice(h->device));
    rc = flush_pending(h);
    if (rc) return rc;
    if (batch == 0) return NLS_OK;
    // candidates are timed on the first S instances; a close final is decided
    // on the first SF (up to the request's size, at most 2^20), where the
    // launch modes' tail effects are those of the real launch
    const int64_t S = std::min<int64_t>(batch, 1 << 18);
    const int64_t SF = std::min<int64_t>(batch, 1 << 20);
    const size_t need = (size_t)n * (size_t)SF * 8 + 256;
    if (need > h->tune_bytes) {
        NLS_CUDA(h, cudaStreamSynchronize(h->stream));
        if (h->d_tune) {
            cudaFree(h->d_tune);
            h->mem_used -= h->tune_bytes;
            h->d_tune = nullptr;
            h->tune_bytes = 0;
        }
        rc = dev_alloc(h, (void **)&h->d_tune, need);
        if (rc) return rc;
        h->tune_bytes = need;
    }
    double *save = h->d_tune; // the first SF instances of u, row pitch SF
    auto *ctr = reinterpret_cast<unsigned long long *>(h->d_tune + (size_t)n * (size_t)SF);
    NLS_CUDA(h, cudaMemcpy2DAsync(save, SF * 8, u, batch * 8, SF * 8, n, cudaMemcpyDeviceToDevice, h->stream));
    const bool mixed = (alg & NLS_MIXED) != 0, analytic = (alg & NLS_ANALYTIC_JAC) != 0;
    std::vector<Tuned> cands;
    auto add = [&](int tiles, int lanes, int refill) {
        Tuned t;
        t.tiles = tiles;
        t.lanes = lanes;
        t.refill = refill;
        cands.push_back(t);
    };
    const bool ext = (alg & NLS_ALG_MASK) >= NLS_POTRA_PTAK;
    if (ext) {
        if (n <= 8)
            for (int r : {REFILL_STATIC, 0, 16, 24, 31}) add(NLS_TILE_THREAD, 0, r);
        for (int r : {REFILL_STATIC, -1}) {
            if (n <= 16) add(NLS_TILE_WARP, 16, r);
            if (n <= 32) add(NLS_TILE_WARP, 32, r);
            if (n > 8) add(NLS_TILE_CTA, 0, r);
        }
    } else if (n <= 8) {
        for (int r : {REFILL_STATIC, 0, 16, 24, 31}) add(NLS_TILE_THREAD, 0, r);
        for (int r : {REFILL_STATIC, -1}) add(NLS_TILE_WARP, 8, r);
    }
    for (int r : {REFILL_STATIC, -1}) {
        if (ext) break;
        if (n <= 16) add(NLS_TILE_WARP, 16, r);
        if (n <= 32) add(NLS_TILE_WARP, 32, r);
        if (n > 8) add(NLS_TILE_CTA, 0, r);
    }
    SolveArgs base{};
    base.params = params;
    base.u = u;
    base.ld = batch;
    base.n = n;
    base.alg = alg & NLS_ALG_MASK;
    base.tr_scheme = (alg & NLS_TR_NOCEDAL_WRIGHT) ? nls::TR_NOCEDAL_WRIGHT : nls::TR_SIMPLE;
    base.abstol = abstol;
    base.maxiters = maxiters;
    // the kernel of a candidate tiling
    auto cand_kernel = [&](const Tuned &c) -> KernelInfo {
        const int a = alg & NLS_ALG_MASK;
        if (ext)
            return c.tiles == NLS_TILE_THREAD ? nls::thread_ext_kernel(family, n, a, mixed)
                   : c.tiles == NLS_TILE_WARP ? nls::warp_ext_kernel(family, c.lanes, a, mixed)
                                              : nls::cta_ext_kernel(family, n, a, mixed);
        return c.tiles == NLS_TILE_THREAD ? thread_kernel(family, n, mixed, analytic)
               : c.tiles == NLS_TILE_WARP ? warp_kernel(family, n, mixed, c.lanes)
                                          : cta_kernel(family, n, mixed);
    };
    Tuned best;
    for (Tuned &c : cands) {
        KernelInfo k = cand_kernel(c);
        if (!k.launch) continue;
        float ms = 0.f;
        rc = tune_trial(h, base, k, c.refill, save, SF, S, ctr, &ms);
        if (rc) return rc;
        c.rate = double(S) / (double(ms) * 1e-3);
        if (c.rate > best.rate) best = c;
    }
    // a close final (within 5%) is decided again, on SF instances: the two
    // leaders alternate for three more best-of-3 rounds, so neither a drift of
    // the clock nor the smaller sample's tail picks the slower launch mode
    {
        std::vector<Tuned *> order;
        for (Tuned &c : cands)
            if (c.rate > 0.0) order.push_back(&c);
        std::sort(order.begin(), order.end(), [](const Tuned *x, const Tuned *y) { return x->rate > y->rate; });
        if (order.size() >= 2 && order[1]->rate > 0.95 * order[0]->rate) {
            Tuned *fin[2] = {order[0], order[1]};
            float bestms[2] = {1e30f, 1e30f};
            for (int round = 0; round < 3; ++round) {
                for (int f = 0; f < 2; ++f) {
                    const Tuned &c = *fin[f];
                    KernelInfo k = cand_kernel(c);
                    float ms = 0.f;
                    rc = tune_trial(h, base, k, c.refill, save, SF, SF, ctr, &ms);
                    if (rc) return rc;
                    bestms[f] = std::min(bestms[f], ms);
                }
            }
            for (int f = 0; f < 2; ++f) fin[f]->rate = double(SF) / (double(bestms[f]) * 1e-3);
            best = fin[0]->rate >= fin[1]->rate ? *fin[0] : *fin[1];
        }
    }
    NLS_CUDA(h, cudaMemcpy2DAsync(u, batch * 8, save, SF * 8, SF * 8, n, cudaMemcpyDeviceToDevice, h->stream));
    NLS_CUDA(h, cudaStreamSynchronize(h->stream));
    h->tuned[tune_key(family, n, alg)] = best;
    if (chosen) *chosen = best.tiles;
    return NLS_OK;
}

int nls_adjoint(nls_handle h, int family, const double *params, const double *u, int n, int64_t batch,
                const double *w, double *grad, int32_t *status)
{
    if (!h) return NLS_E_INVALID;
    if (family < 0 || family > FAM_ROSENBROCK) return fail(h, NLS_E_UNSUPPORTED, "unknown family %d", family);
    if (n < 1 || n > 128) return fail(h, NLS_E_UNSUPPORTED, "nls_adjoint holds n <= 128 (n = %d)", n);
    if (batch < 0) return fail(h, NLS_E_INVALID, "negative batch");
    if (batch == 0) return NLS_OK;
    if (!u || !w) return fail(h, NLS_E_INVALID, "u or w is NULL");
    if (n_params(family, n) > 0 && (!params || !grad)) return fail(h, NLS_E_INVALID, "params or grad is NULL");
    if ((batch + 31) / 32 > INT32_MAX) return fail(h, NLS_E_INVALID, "batch too large");
    NLS_CUDA(h, cudaSetDevice(h->device));
    cudaError_t e = n <= 8 ? nls::launch_adjoint(family, n, params, u, w, grad, status, batch, h->stream)
                           : nls::launch_adjoint_tiles(family, n, params, u, w, grad, status, batch, h->stream);
    if (e != cudaSuccess) return fail(h, NLS_E_CUDA, "adjoint launch: %s", cudaGetErrorString(e));
    ++h->launches;
    return NLS_OK;
}

int nls_tune_lookup(nls_handle h, int family, int n, int alg, int *tiles, int *lanes, int *refill,
                    double *rate)
{
    if (!h) return NLS_E_INVALID;
    auto it = h->tuned.find(tune_key(family, n, alg));
    if (it == h->tuned.end()) return fail(h, NLS_E_NOTFOUND, "no tuned entry for family %d, n = %d", family, n);
    if (tiles) *tiles = it->second.tiles;
    if (lanes) *lanes = it->second.lanes;
    if (refill) *refill = it->second.refill;
    if (rate) *rate = it->second.rate;
    return NLS_OK;
}

int nls_tune_save(nls_handle h, const char *path)
{
    if (!h || !path) return NLS_E_INVALID;
    std::ofstream f(path);
    if (!f) return fail(h, NLS_E_INVALID, "cannot write tuning table %s", path);
    f << "# family n alg tiles lanes refill rate\n";
    for (auto &kv : h->tuned) {
        const long long key = kv.first;
        f << (key >> 40) << ' ' << ((key >> 24) & 0xffff) << ' ' << (key & 0xffffff) << ' ' << kv.second.tiles << ' '
          << kv.second.lanes << ' ' << kv.second.refill << ' ' << kv.second.rate << '\n';
    }
    return f ? NLS_OK : fail(h, NLS_E_INVALID, "writing %s failed", path);
}

int nls_tune_load(nls_handle h, const char *path)
{
    if (!h || !path) return NLS_E_INVALID;
    const int n = load_tuning(h, path);
    return n < 0 ? n : NLS_OK;
}

int nls_set_option(nls_handle h, int option, int64_t value)
{
    if (!h) return NLS_E_INVALID;
    switch (option) {
    case NLS_OPT_PERSISTENT: h->opt.persistent = value != 0; return NLS_OK;
    case NLS_OPT_REFILL_BELOW:
        if (value < 0 || value > 31) return fail(h, NLS_E_INVALID, "refill threshold %lld outside [0, 31]", (long long)value);
        h->opt.refill_below = (int)value;
        return NLS_OK;
    case NLS_OPT_GRAPH: h->opt.graph = value != 0; return NLS_OK;
    case NLS_OPT_DEADLINE_US:
        if (value < 0 || value > (int64_t)1 << 40) return fail(h, NLS_E_INVALID, "deadline %lld us out of range", (long long)value);
        h->opt.deadline_us = value;
        return NLS_OK;
    case NLS_OPT_CTAS_PER_SM:
        if (value < 0 || value > 64) return fail(h, NLS_E_INVALID, "CTAs per SM %lld outside [0, 64]", (long long)value);
        h->opt.ctas_per_sm = (int)value;
        return NLS_OK;
    default: return fail(h, NLS_E_INVALID, "unknown option %d", option);
    }
}

} // extern "C"
