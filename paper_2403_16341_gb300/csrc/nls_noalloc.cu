// nls_noalloc.cu -- nls_solve_noalloc: the thread-tiled batched solve for
// callers that must not allocate device memory.
//
// The persistent solver needs two 64-bit words of global scratch per group
// of instances: the number of solved instances and the work counter its
// warps draw instance ids from.  nls_solve normally keeps them in memory the
// handle allocated; here they live in the file-scope array below, which
// every GPU that loads the library holds until the process exits.  No
// cudaMalloc, cudaFree or other allocating call is made.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "../../include/nls.h"
#include "nls_internal.h"

namespace {

// [2 g] = solved count of group g, [2 g + 1] = its work counter.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[2 * NLS_NOALLOC_MAX_GROUPS];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mu;
unsigned long long *g_scratch_ptr[MAX_DEVICES] = {}; // device address of the array, per device

int err(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int err(int code, const char *fmt, ...)
{
    char buf[384];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return nls::set_global_error(code, buf);
}

// Device address of the scratch array on the current device.  The host-side
// name g_noalloc_scratch is only a stand-in for the symbol, so the address
// is looked up once per device (with that device current) and cached.  The
// cache belongs to the device's primary context (the one the runtime API
// uses): a cudaDeviceReset between calls, or a caller that made another
// context current on that device, would leave a stale address here, and
// neither is supported.
int scratch_on_current_device(unsigned long long **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(NLS_E_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return err(NLS_E_UNSUPPORTED, "device %d out of range", dev);
    std::lock_guard<std::mutex> g(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return err(NLS_E_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        g_scratch_ptr[dev] = static_cast<unsigned long long *>(p);
    }
    *out = g_scratch_ptr[dev];
    return NLS_OK;
}

} // namespace

extern "C" int nls_solve_noalloc(void *cuda_stream, const nls_group *groups, int ngroups, int alg,
                                 double abstol, int maxiters, int64_t *solved)
{
    if (ngroups < 1 || ngroups > NLS_NOALLOC_MAX_GROUPS)
        return err(NLS_E_INVALID,
                   "ngroups = %d: nls_solve_noalloc takes 1..%d groups (its static scratch holds "
                   "%d groups)",
                   ngroups, NLS_NOALLOC_MAX_GROUPS, NLS_NOALLOC_MAX_GROUPS);
    if (!groups) return err(NLS_E_INVALID, "groups is NULL");
    if (!(abstol >= 0.0) || !std::isfinite(abstol)) return err(NLS_E_INVALID, "abstol must be finite and >= 0");
    if (maxiters < 0) return err(NLS_E_INVALID, "negative maxiters");
    if ((alg & NLS_ALG_MASK) > NLS_MOD_BROYDEN) return err(NLS_E_INVALID, "unknown algorithm %d", alg & NLS_ALG_MASK);
    if ((alg & NLS_ALG_MASK) > NLS_TRUST_DOGLEG)
        return err(NLS_E_UNSUPPORTED,
                   "algorithm %d: nls_solve_noalloc runs Newton, backtracking and dogleg only",
                   alg & NLS_ALG_MASK);
    if ((alg & NLS_TR_NOCEDAL_WRIGHT) && (alg & NLS_ALG_MASK) != NLS_TRUST_DOGLEG)
        return err(NLS_E_INVALID, "NLS_TR_NOCEDAL_WRIGHT needs NLS_TRUST_DOGLEG");
    if (alg & ~(NLS_ALG_MASK | NLS_MIXED | NLS_ANALYTIC_JAC | NLS_TILE_THREAD | NLS_TR_NOCEDAL_WRIGHT))
        return err(NLS_E_UNSUPPORTED, "nls_solve_noalloc runs the thread tiling only (flags 0x%x)", alg);
    nls::KernelInfo kern[NLS_NOALLOC_MAX_GROUPS];
    for (int g = 0; g < ngroups; ++g) {
        const nls_group &q = groups[g];
        if (q.n < 1 || q.n > 8)
            return err(NLS_E_UNSUPPORTED, "group %d: n = %d; nls_solve_noalloc supports n <= 8", g, q.n);
        if (q.batch < 0) return err(NLS_E_INVALID, "group %d: negative batch", g);
        const bool np = q.family == NLS_ROSENBROCK;
        if (q.batch > 0 && (!q.u || (!np && !q.params)))
            return err(NLS_E_INVALID, "group %d: NULL params or u", g);
        kern[g] = nls::thread_kernel(q.family, q.n, (alg & NLS_MIXED) != 0, (alg & NLS_ANALYTIC_JAC) != 0);
        if (!kern[g].launch) return err(NLS_E_UNSUPPORTED, "group %d: unknown family %d", g, q.family);
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (solved) {
        // reading the counts back waits for the stream, which a capture forbids
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        cudaError_t ce = cudaStreamIsCapturing(st, &cap);
        if (ce != cudaSuccess) return err(NLS_E_CUDA, "cudaStreamIsCapturing: %s", cudaGetErrorString(ce));
        if (cap != cudaStreamCaptureStatusNone)
            return err(NLS_E_INVALID, "solved must be NULL while the stream is being captured");
    }
    unsigned long long *scratch = nullptr;
    int rc = scratch_on_current_device(&scratch);
    if (rc) return rc;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // the counters must start at zero: the previous call left its totals here
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * 2 * ngroups, st);
    if (e != cudaSuccess) return err(NLS_E_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    for (int g = 0; g < ngroups; ++g) {
        const nls_group &q = groups[g];
        if (q.batch == 0) continue;
        nls::SolveArgs a{};
        a.params = q.params;
        a.u = q.u;
        a.batch = q.batch;
        a.ld = q.batch;
        a.n = q.n;
        a.alg = alg & NLS_ALG_MASK;
        a.tr_scheme = (alg & NLS_TR_NOCEDAL_WRIGHT) ? nls::TR_NOCEDAL_WRIGHT : nls::TR_SIMPLE;
        a.abstol = abstol;
        a.maxiters = maxiters;
        a.status = q.out.status;
        a.iters = q.out.iters;
        a.resid = q.out.resid_inf;
        a.nfev = q.out.nfev;
        a.ngrad = q.out.ngrad;
        a.solved = scratch + 2 * g;
        a.counter = scratch + 2 * g + 1;
        a.refill_below = 24;
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern[g].func, kern[g].block, kern[g].smem);
        if (e != cudaSuccess) return err(NLS_E_CUDA, "occupancy query: %s", cudaGetErrorString(e));
        const int64_t ctas = (q.batch + kern[g].per_cta - 1) / kern[g].per_cta;
        const int grid = (int)std::min<int64_t>(ctas, (int64_t)std::max(occ, 1) * sms);
        e = kern[g].launch(a, grid, st);
        if (e != cudaSuccess) return err(NLS_E_CUDA, "kernel launch: %s", cudaGetErrorString(e));
    }
    if (solved) {
        unsigned long long host[2 * NLS_NOALLOC_MAX_GROUPS];
        e = cudaMemcpyAsync(host, scratch, sizeof(unsigned long long) * 2 * ngroups, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return err(NLS_E_CUDA, "reading the solved counts: %s", cudaGetErrorString(e));
        for (int g = 0; g < ngroups; ++g) solved[g] = (int64_t)host[2 * g];
    }
    return NLS_OK;
}
