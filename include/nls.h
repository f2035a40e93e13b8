/*
 * nls.h -- C ABI of the GB300 batched small-system nonlinear solver.
 *
 * The library solves very many small, independent nonlinear systems
 *
 *     find u*_k  such that  F(u*_k; p_k) = 0,   k = 0 .. batch-1,
 *
 * (the problem statement of Sec. 2, Eq. 1, with theta = p_k), each instance
 * with Newton-Raphson (Sec. 2.1, Eq. 2), Newton-Raphson with a backtracking
 * line search (Sec. 2.2.1, Eq. 8-9) or a trust region with Powell's dogleg
 * step (Sec. 2.2.2, Eq. 13-15); or with Halley's method (Sec. 2.1, Eq. 3),
 * the Potra-Ptak two-step method (Sec. 2.1, Eq. 4), Broyden's quasi-Newton
 * method (Sec. 3.1, Tab. 1), or the poly-algorithm that chains them
 * (Sec. 3.2).  The Jacobian comes from forward-mode dual numbers (Sec. 2.4)
 * or from the family's analytic formula, and each Newton system is solved
 * with a dense LU with partial pivoting (Sec. 3.2, Fig. 5).  nls_adjoint
 * returns the sensitivity of the roots to the parameters (Sec. 2.3).
 * An instance has converged when ||F(u_k)||_inf <= abstol (Sec. 2.1).  The
 * paper's own GPU form of this path is Sec. 3.3: statically sized,
 * non-allocating solvers, one instance per GPU thread.
 *
 * Conventions for every call:
 *   - Every function returns an nls_err (0 = NLS_OK, negative = error) and,
 *     on error, leaves a message for nls_last_error().  Argument errors are
 *     detected before anything is enqueued.
 *   - Device pointers are CUDA device (or managed) addresses on the handle's
 *     device; they stay owned by the caller and must stay valid until the
 *     request has completed (nls_status returns NLS_OK for it).
 *   - Per-instance failures (singular Jacobian, NaN, no convergence) are
 *     never API errors: they are reported per instance as nls_inst_status.
 *   - A handle is not thread-safe: use one handle per host thread or lock.
 *
 * Batch layout ("SoA", element-major, instance fastest): element e of
 * instance k is at ptr[e * batch + k].  Parameters per family (E values):
 *   NLS_CUBIC      F = A u + u.*u.*u - b:  e = i*n + j -> A[i][j]
 *                  (row-major), e = n*n + i -> b[i];          E = n*n + n
 *   NLS_BRATU      F_i = (u_{i-1} - 2 u_i + u_{i+1}) (n+1)^2 + lambda e^{u_i},
 *                  u_0 = u_{n+1} = 0 (1-D Bratu, h = 1/(n+1)): e = 0 -> lambda; E = 1
 *   NLS_SQUARE     F = u.*u - p (the Sec. 2.3 example):  e = i -> p[i];   E = n
 *   NLS_ROSENBROCK generalized Rosenbrock (Sec. 2.2.1, Eq. 5): no parameters, E = 0
 */
#ifndef NLS_H
#define NLS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nls_batch *nls_handle; /* opaque, owned by the library */

enum nls_family { NLS_CUBIC = 0, NLS_BRATU = 1, NLS_SQUARE = 2, NLS_ROSENBROCK = 3 };

/* Algorithm in the low byte of `alg`; flags are OR-ed in. */
enum nls_alg {
    NLS_NEWTON = 0,           /* Sec. 2.1, Eq. 2                               */
    NLS_NEWTON_BACKTRACK = 1, /* Sec. 2.2.1: Armijo (Eq. 8-9), alpha <- alpha/2 */
    NLS_TRUST_DOGLEG = 2,     /* Sec. 2.2.2: Eq. 13-15, Powell's dogleg          */
    NLS_POLYALG = 3,          /* Sec. 3.2 poly-algorithm: the first stage runs
                                 on every instance, the ones that fail
                                 restart from u0 with the next stage.  n > 25:
                                 Broyden, modified Broyden (the quasi-Newton
                                 phase; Klement is not built), Newton,
                                 backtracking, trust region; n <= 25: Newton,
                                 backtracking, trust region (the paper skips
                                 quasi-Newton there).  iters = the final
                                 stage's passes, nfev = all stages' residual
                                 evaluations.                                 */
    /* The following take forward-mode derivatives only (NLS_ANALYTIC_JAC:
       NLS_E_UNSUPPORTED) and run on every tiling (n <= 128). */
    NLS_POTRA_PTAK = 4,       /* Sec. 2.1, Eq. 4: y = u + du1, u' = y + du2 with
                                 J(u) du1 = -F(u), J(u) du2 = -F(y) (one
                                 Jacobian and LU, two residuals per pass)     */
    NLS_HALLEY = 5,           /* Sec. 2.1, Eq. 3: a = -J^-1 F, J b = H a a
                                 (second directional derivative by forward-
                                 mode jets), step (a o a) / (a + b/2)
                                 elementwise; a_i where a_i + b_i/2 == 0      */
    NLS_BROYDEN = 6,          /* Sec. 3.1, Tab. 1: quasi-Newton, B_0 = I, good
                                 Broyden update after each full step; kept as
                                 B^-1 (Sherman-Morrison), no Jacobian, no LU.
                                 A singular update ends NLS_SINGULAR.         */
    NLS_MOD_BROYDEN = 7       /* Tab. 1 "Mod. Broyden": as NLS_BROYDEN with
                                 B_0 = J(u_0) by forward mode                  */
};
#define NLS_ALG_MASK 0xff
enum nls_flags {
    NLS_MIXED = 1 << 8,        /* Jacobian + LU in FP32; residual, norm test,
                                  merit and update in FP64                      */
    NLS_ANALYTIC_JAC = 1 << 9, /* family's closed-form Jacobian instead of duals */
    NLS_TILE_THREAD = 1 << 10, /* force one instance per thread   (n <= 8)      */
    NLS_TILE_WARP = 1 << 11,   /* force one instance per warp     (n <= 32)     */
    NLS_TILE_CTA = 1 << 12,    /* force one instance per CTA      (n <= 128)    */
    NLS_TR_NOCEDAL_WRIGHT = 1 << 13, /* trust-region radius update of Tab. 3's
                                  NocedalWright scheme (Nocedal & Wright,
                                  Algorithm 4.1): shrink x1/4 iff rho < 1/4,
                                  double (cap 1e3) iff rho > 3/4 and the step
                                  reached the boundary, accept iff
                                  rho > 1e-4.  Without it: accept iff rho > 0,
                                  double iff rho > 3/4, shrink x1/4 on
                                  rejection.  Valid with NLS_TRUST_DOGLEG and
                                  NLS_POLYALG (its trust-region stage).      */
    NLS_REFINE = 1 << 14       /* with NLS_MIXED: classical iterative
                                  refinement of every Newton step (the second
                                  reading of "FP32 LU with FP64 residual
                                  refinement" for n up to 128): after the
                                  FP32 LU gives dN, two passes of
                                  r = -F - J dN with J in FP64 (evaluated on
                                  the fly, no FP64 copy of J is stored) and
                                  dN += the FP32 factors' solve of r.  Runs
                                  on the CTA tiling (any n <= 128) with
                                  NLS_NEWTON, NLS_NEWTON_BACKTRACK and
                                  NLS_TRUST_DOGLEG; other combinations, and
                                  nls_autotune, return NLS_E_UNSUPPORTED.   */
};

/* Per-instance outcome. */
enum nls_inst_status {
    NLS_SUCCESS = 0,    /* ||F(u)||_inf <= abstol                               */
    NLS_MAXITERS = 1,   /* maxiters passes without convergence                   */
    NLS_SINGULAR = 2,   /* an LU pivot was exactly zero or not finite            */
    NLS_NONFINITE = 3,  /* F became Inf/NaN (at u0, or after an accepted step)   */
    NLS_LS_FAILED = 4,  /* 30 backtracking trials without sufficient decrease    */
    NLS_TR_STALLED = 5, /* 32 trust-region rejections in a row                   */
    NLS_ABORTED = 6     /* the launch's deadline (NLS_OPT_DEADLINE_US) passed
                           before convergence; u holds the last iterate        */
};

enum nls_err {
    NLS_OK = 0,
    NLS_E_INVALID = -1,     /* bad argument (null pointer, negative size, ...)  */
    NLS_E_CUDA = -2,        /* a CUDA runtime call failed                       */
    NLS_E_NOMEM = -3,       /* workspace would exceed the memory cap            */
    NLS_E_UNSUPPORTED = -4, /* n outside [1, 128], unknown family or tiling     */
    NLS_E_TIMEOUT = -5,     /* the request did not complete within timeout_ms   */
    NLS_E_BUSY = -6,        /* the handle is inside another operation           */
    NLS_E_NOTFOUND = -7     /* unknown request id                               */
};

/* Fixed algorithm constants (the paper gives no values; see nls_oracle.c
 * for the same readings):
 *   backtracking c1 = 1e-4, step factor 1/2, at most 30 trials;
 *   trust region Delta_0 = 1, accept iff rho > 0, grow x2 (cap 1e3) iff
 *   rho > 0.75, on rejection shrink x1/4; 32 rejections in a row stall. */

/* Per-instance outputs (all DEVICE pointers, each may be NULL = not written):
 * status[k] (nls_inst_status), iters[k] (loop passes), resid_inf[k] =
 * ||F(u_k)||_inf of the returned u_k in FP64, nfev[k] = FP64 residual
 * evaluations used, ngrad[k] = trust-region passes that formed the dogleg's
 * gradient g = J^T F and J g (Eq. 13-14; the thread tiling forms them only
 * when the Newton step leaves the region, the warp and CTA tilings with
 * every new Jacobian); 0 for the other algorithms and for NLS_POLYALG. */
typedef struct nls_outputs {
    int32_t *status;
    int32_t *iters;
    double *resid_inf;
    int32_t *nfev;
    int32_t *ngrad;
} nls_outputs;

/* Create a solver context on `device` that enqueues on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  mem_cap_bytes bounds
 * the library-owned device workspace (0 = no cap beyond free memory).  That
 * workspace is small and grows on demand: a ring of 64 Ki 64-bit counters,
 * the staging buffers of nls_solve_host, the autotuner's scratch and the
 * poly-algorithm's gather buffers; the caller's own arrays are never
 * counted.  (The request server, which holds request state, admits by free
 * device memory minus a reserve instead: nls_server_create.)
 * Errors: NLS_E_INVALID (out == NULL), NLS_E_CUDA (bad device). */
int nls_batch_create(nls_handle *out, int device, void *cuda_stream, size_t mem_cap_bytes);

/* Enqueue the solve of `batch` instances of `family` with size n
 * (Sec. 2, Eq. 1).  params: DEVICE float64[E * batch] (may be NULL when
 * E = 0); u: DEVICE float64[n * batch], read as u0 and overwritten with the
 * returned iterate; out: optional per-instance outputs (NULL = none).
 * alg = nls_alg | nls_flags.  abstol >= 0 (finite), maxiters >= 0.
 * Requests are grouped until nls_flush or nls_status, which launch every
 * pending request of the handle together in one CUDA-graph launch: a lone
 * request as a persistent kernel (work counter, idle lanes refilled), several
 * requests as concurrent kernel nodes with full grids whose blocks the
 * hardware interleaves.  *req receives an id for nls_status.
 * batch == 0 is a no-op that still returns an id.
 * Errors: NLS_E_INVALID (null pointers, negative batch/maxiters, bad abstol,
 * unknown algorithm or flag), NLS_E_UNSUPPORTED (n outside [1, 128], unknown
 * family, tiling that cannot hold n, a flag the algorithm does not take:
 * NLS_ANALYTIC_JAC with NLS_POTRA_PTAK..NLS_MOD_BROYDEN, NLS_REFINE outside
 * NLS_MIXED Newton / backtracking / trust region on the CTA tiling). */
int nls_solve(nls_handle h, int family, const double *params, double *u, int n, int64_t batch,
              int alg, double abstol, int maxiters, const nls_outputs *out, int64_t *req);

/* Sensitivity of the roots to the parameters (Sec. 2.3, implicit function
 * theorem).  At roots u (DEVICE float64[n * batch], e.g. from nls_solve) with
 * J = dF/du, du/dtheta = -J^{-1} dF/dtheta; for cotangents w = dL/du (DEVICE
 * float64[n * batch]) this computes, per instance, mu from J^T mu = w and
 * grad = dL/dtheta = -mu^T dF/dtheta (DEVICE float64[E * batch], the family's
 * parameter layout).  status (DEVICE int32[batch], may be NULL) receives
 * NLS_SUCCESS or NLS_SINGULAR.  FP64, forward-mode Jacobian; one instance
 * per thread (n <= 8), per warp segment (n <= 32) or per CTA (n <= 128).
 * Enqueued on the handle's stream at once (not grouped with nls_solve
 * requests); order it after the solve that produced u.
 * Errors: NLS_E_INVALID, NLS_E_UNSUPPORTED (n > 128, unknown family),
 * NLS_E_CUDA. */
int nls_adjoint(nls_handle h, int family, const double *params, const double *u, int n,
                int64_t batch, const double *w, double *grad, int32_t *status);

/* Launch every pending request of the handle on its stream (asynchronous). */
int nls_flush(nls_handle h);

/* Completion of request `req`: flushes if needed, then waits up to
 * timeout_ms on the host (< 0 = no limit, 0 = poll; the device never
 * waits).  On NLS_OK, *solved (may be NULL) = number of its instances with
 * status NLS_SUCCESS.  NLS_E_TIMEOUT if not complete yet (query again);
 * NLS_E_NOTFOUND for an unknown or already released id.
 * The per-instance status, iters, resid_inf (and nfev) are not passed here:
 * they are bound when the request is made (nls_solve's `out`), so the
 * kernels write them straight into the caller's arrays, with no library
 * copy, and they are complete once this call returns NLS_OK. */
int nls_status(nls_handle h, int64_t req, int64_t *solved, int timeout_ms);

/* Synchronous end-to-end variant on HOST buffers: copies params and u
 * (pinned host memory is fastest) into library-owned device memory, solves,
 * copies u and the per-instance outputs (HOST pointers in `out`, each may be
 * NULL) back, and waits.  Batches of 2^18 instances and more (not
 * NLS_POLYALG) are pipelined in up to eight chunks: a chunk's upload, solve
 * and download overlap the neighbouring chunks', and consecutive chunks'
 * solves run on two alternating streams of the handle, so one chunk's
 * launch fills the SMs the previous chunk's grid frees as it drains.
 * Requests made earlier with nls_solve and not yet launched are launched
 * first, on the handle's stream.  Same arguments and errors as nls_solve,
 * plus NLS_E_NOMEM when the staging buffers would exceed the memory cap. */
int nls_solve_host(nls_handle h, int family, const double *params, double *u, int n,
                   int64_t batch, int alg, double abstol, int maxiters, const nls_outputs *out,
                   int64_t *solved);

/* Asynchronous form of nls_solve_host: enqueues the uploads, the solve and
 * the downloads on the handle's streams and returns at once with a request
 * id in *req; nls_status(h, *req, ...) waits for it (the results are then in
 * the host buffers and *solved counts the NLS_SUCCESS instances).  params,
 * u and the host outputs must stay valid, and must not be written, until
 * nls_status has returned NLS_OK for the id.  Requests made one after
 * another run as a pipeline: the next request's uploads overlap the current
 * request's solve, its solve the current request's downloads.  Each request
 * in flight holds its own library-owned staging block (about the size of its
 * device state); blocks are reused by later requests.  Same arguments and
 * errors as nls_solve_host (plus NLS_E_INVALID for req == NULL). */
int nls_solve_host_async(nls_handle h, int family, const double *params, double *u, int n,
                         int64_t batch, int alg, double abstol, int maxiters,
                         const nls_outputs *out, int64_t *req);

/* Destroy the context; waits for its outstanding work first. */
int nls_batch_destroy(nls_handle h);

/* Message of the last error on this handle (or of a failed create when
 * h == NULL); never NULL. */
const char *nls_last_error(nls_handle h);

/* Kernels launched by this handle since creation (for launch accounting). */
int64_t nls_launch_count(nls_handle h);

/* Scheduling options of a handle (apply to later flushes). */
enum nls_option {
    NLS_OPT_PERSISTENT = 1,   /* 1 (default): persistent grid of about one wave
                                 of CTAs pulling instances from a work counter;
                                 0: one CTA per block of instances             */
    NLS_OPT_REFILL_BELOW = 2, /* thread tiling, persistent: a warp refills its
                                 idle lanes when at most this many lanes are
                                 still iterating (0..31, default 24)           */
    NLS_OPT_CTAS_PER_SM = 3,  /* cap on resident CTAs per SM (0 = occupancy)   */
    NLS_OPT_DEADLINE_US = 5,  /* > 0: each launch stops iterating this many
                                 microseconds (device clock) after it starts;
                                 unfinished instances end NLS_ABORTED.  0 (the
                                 default): no deadline.  Applies to requests
                                 enqueued afterwards.                          */
    NLS_OPT_GRAPH = 4         /* 1 (default): a flush is one CUDA-graph launch
                                 (counter reset, one kernel node per request,
                                 all concurrent, counter read-back), cached by
                                 the shape of the group; 0: direct launches    */
};
/* Errors: NLS_E_INVALID for an unknown option or a value out of range. */
int nls_set_option(nls_handle h, int option, int64_t value);

/* Autotuner: times each tiling that can hold n -- thread (n <= 8), warp with
 * 8, 16 or 32 lanes (n <= lanes), CTA (n > 8) -- each both as a persistent
 * grid (thread tiling: refill thresholds 0/16/24/31) and as a
 * one-block-per-chunk grid (best of three runs), on the first min(batch, 2^18) instances of this
 * batch; when the two fastest are within 5%, they are timed again,
 * alternately, on the first min(batch, 2^20) instances.  Keeps the fastest
 * for (family, n, algorithm, precision) in the
 * handle's table and restores u.  Later nls_solve calls without a tiling
 * flag use the table (a request flushed alone takes the tuned launch mode;
 * requests flushed together always use one-block-per-chunk grids).
 * Synchronous.  Same arguments as nls_solve (no tiling flag allowed);
 * *chosen (may be NULL) receives the chosen NLS_TILE_* flag.  If the
 * environment variable NLS_TUNE_CACHE names a file when a handle is created,
 * the table is read from it. */
int nls_autotune(nls_handle h, int family, const double *params, double *u, int n, int64_t batch,
                 int alg, double abstol, int maxiters, int *chosen);
/* The tuned entry for (family, n, alg): tiling flag, warp lanes, refill
 * (-2 one-block-per-chunk grid, -1 persistent with the handle's threshold,
 * >= 0 persistent with that threshold) and the measured instances/s.
 * NLS_E_NOTFOUND when (family, n, alg) has not been tuned. */
int nls_tune_lookup(nls_handle h, int family, int n, int alg, int *tiles, int *lanes, int *refill,
                    double *rate);
/* Write / read the tuning table (text: family n alg tiles lanes refill rate;
 * refill -2 = one-block-per-chunk grid, -1 = persistent with the handle's
 * threshold, >= 0 = persistent with that threshold). */
int nls_tune_save(nls_handle h, const char *path);
int nls_tune_load(nls_handle h, const char *path);

/* ------------------------------------------------------------------------
 * Request server (continuous batching).
 *
 * Serves solve requests that arrive over time, each a batch of instances of
 * one (family, n) on HOST buffers (pinned memory is fastest).  A dispatcher
 * thread admits waiting requests in arrival order as soon as their device
 * state fits in the server's arena (a block of device memory of
 * mem_budget_bytes, 0 = half of the free memory; never more than free memory
 * minus 1 GiB), copies their inputs in, and launches each wave of admitted
 * requests through one of `streams` worker handles, so that waves admitted
 * while others run overlap on the GPU.  Results (u and the per-instance
 * outputs) are copied back into the caller's host buffers; then the arena
 * space is released and waiting requests are admitted.  Each instance is
 * solved exactly as by nls_solve with the same arguments.  The server is
 * thread-safe: any thread may submit and wait. */
typedef struct nls_server *nls_server_t;
/* Errors: NLS_E_INVALID (streams outside 1..16), NLS_E_NOMEM, NLS_E_CUDA. */
int nls_server_create(nls_server_t *out, int device, size_t mem_budget_bytes, int streams);
/* Queue a request.  params / u / out are HOST pointers that must stay valid
 * until nls_server_wait returns for the ticket; u holds u0 and receives the
 * roots.  Same argument rules as nls_solve; NLS_E_NOMEM if the request can
 * never fit in the arena. */
int nls_server_submit(nls_server_t s, int family, const double *params, double *u, int n,
                      int64_t batch, int alg, double abstol, int maxiters, const nls_outputs *out,
                      int64_t *ticket);
/* Wait (timeout_ms < 0: no limit) for a ticket; on NLS_OK its results are in
 * the host buffers, *solved = #NLS_SUCCESS, *t_submit / *t_done = server
 * clock (seconds, see nls_server_now) of submission and of the results
 * being on the host.  The ticket is released. */
int nls_server_wait(nls_server_t s, int64_t ticket, int64_t *solved, double *t_submit,
                    double *t_done, int timeout_ms);
/* Where a request's time went, for latency analysis.  Host times are on the
 * server clock (seconds, nls_server_now); device times come from CUDA events
 * on the request's worker stream (-1 where they could not be taken).  A wave
 * is the group of requests one dispatcher round admitted onto one worker
 * stream: their inputs are copied in, then solved by one flush. */
typedef struct nls_server_timing {
    double t_submit;   /* nls_server_submit returned the ticket              */
    double t_admit;    /* the dispatcher admitted it (its state fit)         */
    double t_launch;   /* its wave's copies and solve were enqueued          */
    double t_done;     /* the dispatcher saw its results in host memory      */
    float h2d_ms;      /* device time of its wave's host-to-device copies    */
    float solve_ms;    /* from the end of those copies to the end of its
                          wave's flush on the stream: the host's enqueue of
                          the wave's requests, then the solve              */
    float d2h_ms;      /* from the end of that solve to its results copied   */
    int wave_requests; /* requests in its wave                               */
} nls_server_timing;
/* nls_server_wait with the request's stage times in *timing (may be NULL). */
int nls_server_wait_timed(nls_server_t s, int64_t ticket, int64_t *solved,
                          nls_server_timing *timing, int timeout_ms);
/* Seconds since the server was created (monotonic clock). */
double nls_server_now(nls_server_t s);
/* Counters: admitted, completed, solved instances, max queue depth, max
 * requests in flight, launch waves, queue depth, in flight, arena bytes,
 * largest free arena block (the first ncounters of these). */
int nls_server_stats(nls_server_t s, int64_t *counters, int ncounters);
/* Finish all queued and in-flight work, then free the server. */
int nls_server_destroy(nls_server_t s);

/* ------------------------------------------------------------------------
 * Allocation-free solve (the paper has no counterpart).
 *
 * For callers that cannot allocate device memory: code running inside
 * another runtime that owns all of the GPU's memory (a plug-in or custom
 * call of a framework with its own pool, a simulator with a fixed arena),
 * or a hot path that cannot afford cudaMalloc's implicit device-wide
 * synchronisation.  It needs no handle and makes no cudaMalloc, cudaFree,
 * cudaMallocHost or other allocating call.
 *
 * Solves up to NLS_NOALLOC_MAX_GROUPS groups, each of one (family, n) with
 * n <= 8, with the persistent thread-tiled kernel of nls_solve.  It runs
 * Newton, backtracking and the dogleg trust region (with NLS_MIXED,
 * NLS_ANALYTIC_JAC and NLS_TR_NOCEDAL_WRIGHT as for nls_solve); the other
 * algorithms of nls_solve give NLS_E_UNSUPPORTED here.  Each group
 * needs two 64-bit counters (its work counter and its solved count); they
 * live in one static device array of NLS_NOALLOC_MAX_GROUPS * 16 bytes that
 * every GPU loading the library holds until the process exits.  All calls
 * share that array and reset the counters they use at the start of the
 * call, so calls that overlap on the GPU (two streams, two host threads)
 * race: serialise them.  The first call on a device looks up the array's
 * device address and caches it; make that first call before any stream
 * capture.  The cached address belongs to the device's primary context:
 * calls after a cudaDeviceReset, or from another context made current on
 * the same device, are not supported.  A call on a stream that is being
 * captured must pass solved = NULL (reading the counts waits for the
 * stream); otherwise it returns NLS_E_INVALID with nothing enqueued.
 *
 * Runs on the current device, enqueued on cuda_stream (NULL = legacy
 * default stream).  Inputs and outputs are the caller's DEVICE pointers,
 * laid out as for nls_solve.  If `solved` (HOST int64[ngroups]) is not
 * NULL the call waits for the stream and stores each group's number of
 * NLS_SUCCESS instances; with NULL it returns once everything is enqueued.
 * Errors: NLS_E_INVALID (ngroups outside 1..NLS_NOALLOC_MAX_GROUPS, NULL
 * pointers, bad abstol / maxiters, an unknown algorithm, solved != NULL
 * during a capture), NLS_E_UNSUPPORTED (n > 8, unknown family, a warp or
 * CTA tiling flag, an algorithm other than the three above), NLS_E_CUDA;
 * the message is in nls_last_error(NULL). */
#define NLS_NOALLOC_MAX_GROUPS 64
typedef struct nls_group {
    int family;
    int n;
    const double *params; /* DEVICE float64[E * batch] */
    double *u;            /* DEVICE float64[n * batch], u0 in, iterate out */
    int64_t batch;
    nls_outputs out;      /* optional DEVICE outputs, as for nls_solve */
} nls_group;
int nls_solve_noalloc(void *cuda_stream, const nls_group *groups, int ngroups, int alg,
                      double abstol, int maxiters, int64_t *solved);

#ifdef __cplusplus
}
#endif
#endif /* NLS_H */
