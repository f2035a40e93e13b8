// nls_internal.h -- host-side registry of the solver kernels.
#pragma once

#include <cuda_runtime.h>

#include "nls_common.cuh"

namespace nls {

using LaunchFn = cudaError_t (*)(const SolveArgs &, int grid, cudaStream_t);

struct KernelInfo {
    LaunchFn launch = nullptr;
    const void *func = nullptr;
    int block = 0;     // threads per CTA
    int smem = 0;      // dynamic shared memory bytes
    int per_cta = 0;   // instances per CTA per round (static grids)
};

// One instance per thread, compile-time n in 1..8.
KernelInfo thread_kernel(int family, int n, bool mixed, bool analytic);

// Record a handle-free error message for nls_last_error(NULL); returns code.
int set_global_error(int code, const char *msg);

} // namespace nls

namespace nls {
// One instance per warp segment of L = 8, 16 or 32 lanes (the smallest L >= n,
// or `lanes` when non-zero), runtime n <= L.
KernelInfo warp_kernel(int family, int n, bool mixed, int lanes = 0);
} // namespace nls

namespace nls {
// One instance per CTA, n <= 128.  Mixed precision: the column-panel solver
// (nls_panel.cuh, 16 columns of J per warp); FP64: the 256-thread CTA with
// R x R block-cyclic register tiles (nls_cta.cuh, R = 4: n <= 64, 8: n <= 128).
KernelInfo cta_kernel(int family, int n, bool mixed);
} // namespace nls

namespace nls {
// Adjoint sensitivity kernels: one instance per thread (n <= 8), ...
cudaError_t launch_adjoint(int family, int n, const double *params, const double *u, const double *w,
                           double *grad, int32_t *status, int64_t batch, cudaStream_t st);
// ... per warp segment (n <= 32) or per CTA (n <= 128).
cudaError_t launch_adjoint_tiles(int family, int n, const double *params, const double *u, const double *w,
                                 double *grad, int32_t *status, int64_t batch, cudaStream_t st);
} // namespace nls

namespace nls {
// Poly-algorithm helpers (nls_poly.cu).
struct PolyGatherArgs {
    int64_t batch;               // full batch (also the compact arrays' leading dimension)
    int E, n;
    const int32_t *status;       // [batch] statuses after the previous stage
    const double *params;        // [E][batch]
    const double *u0;            // [n][batch] original starting points
    int64_t *idx;                // [batch] compact position -> instance
    double *cparams, *cu;        // [E][batch], [n][batch] compact copies
    unsigned long long *count;   // number gathered (zeroed before)
};
struct PolyScatterArgs {
    int64_t batch;
    int n;
    const unsigned long long *count;
    const int64_t *idx;
    const double *cu;
    const int32_t *cstatus, *citers, *cnfev;
    const double *cresid;
    double *u;
    int32_t *status, *iters, *nfev;
    double *resid;
};
cudaError_t launch_poly_gather(const PolyGatherArgs &g, cudaStream_t st);
cudaError_t launch_poly_scatter(const PolyScatterArgs &s, cudaStream_t st);
cudaError_t launch_poly_total(unsigned long long *solved, const unsigned long long *ctr, int stages,
                              cudaStream_t st);
// Potra-Ptak, Halley, Broyden and modified Broyden (alg = ALG_POTRA_PTAK ..
// ALG_MOD_BROYDEN): one instance per thread (n <= 8), per warp segment of
// L = 16 or 32 lanes, or per CTA (n <= 128).
KernelInfo thread_ext_kernel(int family, int n, int alg, bool mixed);
KernelInfo warp_ext_kernel(int family, int L, int alg, bool mixed);
KernelInfo cta_ext_kernel(int family, int n, int alg, bool mixed);
} // namespace nls
