// nls_adjoint.cu -- sensitivity of the roots to the parameters (Sec. 2.3).
//
// At a root u* of F(u; theta) = 0 the implicit function theorem gives
// du*/dtheta = -J^{-1} dF/dtheta with J = dF/du at u* (the printed formula
// drops the minus sign).  For a loss with cotangent w = dL/du*, the adjoint
// form needs one transposed solve per instance instead of one solve per
// parameter:  J^T mu = w,  dL/dtheta = -mu^T dF/dtheta.
// One instance per thread (n <= 8): the dual-number Jacobian and the
// register LU of the solver, applied to J^T, all in FP64.
#include <cuda_runtime.h>

#include "../../include/nls.h"
#include "nls_internal.h"
#include "nls_thread.cuh"

namespace nls {

struct AdjointArgs {
    const double *params; // [E][batch]
    const double *u;      // [n][batch] roots
    const double *w;      // [n][batch] dL/du
    double *grad;         // [E][batch] dL/dtheta
    int32_t *status;      // [batch] NLS_SUCCESS or NLS_SINGULAR (may be null)
    int64_t batch;
};

template <int N, int FAM>
__global__ void __launch_bounds__(THREAD_TPB) k_adjoint_thread(AdjointArgs a)
{
    using S = ThreadSolver<N, FAM, false, false>;
    constexpr int E = S::E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *sd = reinterpret_cast<double *>(smem_raw);
    const int lane = threadIdx.x;
    const int64_t k = (int64_t)blockIdx.x * THREAD_TPB + lane;
    if (k >= a.batch) return;
    const int64_t B = a.batch;
#pragma unroll 4
    for (int e = 0; e < E; ++e) sd[e * THREAD_TPB + lane] = __ldg(a.params + (int64_t)e * B + k);
    const ParamView pv{sd + lane, nullptr, THREAD_TPB};
    double u[N], J[N][N], Jt[N][N], mu[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        u[i] = a.u[(int64_t)i * B + k];
        mu[i] = a.w[(int64_t)i * B + k];
    }
    S::jacobian(pv, u, J);
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) Jt[i][j] = J[j][i];
    const bool ok = lu_solve<N, double>(Jt, mu); // mu = J^-T w
    if (a.status) a.status[k] = ok ? ST_SUCCESS : ST_SINGULAR;
    if constexpr (FAM == FAM_CUBIC) {
        // dF_i/dA_ij = u_j, dF_i/db_i = -1
#pragma unroll
        for (int i = 0; i < N; ++i) {
#pragma unroll
            for (int j = 0; j < N; ++j) a.grad[(int64_t)(i * N + j) * B + k] = -mu[i] * u[j];
            a.grad[(int64_t)(N * N + i) * B + k] = mu[i];
        }
    } else if constexpr (FAM == FAM_BRATU) {
        // dF_i/dlambda = exp(u_i)
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < N; ++i) s = fma(mu[i], exp(u[i]), s);
        a.grad[k] = -s;
    } else if constexpr (FAM == FAM_SQUARE) {
        // dF_i/dp_i = -1
#pragma unroll
        for (int i = 0; i < N; ++i) a.grad[(int64_t)i * B + k] = mu[i];
    }
}

template <int N, int FAM>
static cudaError_t launch_adjoint_n(const AdjointArgs &a, cudaStream_t st)
{
    const int64_t grid = (a.batch + THREAD_TPB - 1) / THREAD_TPB;
    const int smem = THREAD_TPB * family_params<FAM>(N) * 8;
    k_adjoint_thread<N, FAM><<<(unsigned)grid, THREAD_TPB, smem, st>>>(a);
    return cudaGetLastError();
}

template <int FAM>
static cudaError_t launch_adjoint_f(int n, const AdjointArgs &a, cudaStream_t st)
{
    switch (n) {
    case 1: return launch_adjoint_n<1, FAM>(a, st);
    case 2: return launch_adjoint_n<2, FAM>(a, st);
    case 3: return launch_adjoint_n<3, FAM>(a, st);
    case 4: return launch_adjoint_n<4, FAM>(a, st);
    case 5: return launch_adjoint_n<5, FAM>(a, st);
    case 6: return launch_adjoint_n<6, FAM>(a, st);
    case 7: return launch_adjoint_n<7, FAM>(a, st);
    case 8: return launch_adjoint_n<8, FAM>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_adjoint(int family, int n, const double *params, const double *u, const double *w,
                           double *grad, int32_t *status, int64_t batch, cudaStream_t st)
{
    AdjointArgs a{params, u, w, grad, status, batch};
    switch (family) {
    case FAM_CUBIC: return launch_adjoint_f<FAM_CUBIC>(n, a, st);
    case FAM_BRATU: return launch_adjoint_f<FAM_BRATU>(n, a, st);
    case FAM_SQUARE: return launch_adjoint_f<FAM_SQUARE>(n, a, st);
    case FAM_ROSENBROCK: return launch_adjoint_f<FAM_ROSENBROCK>(n, a, st);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace nls
