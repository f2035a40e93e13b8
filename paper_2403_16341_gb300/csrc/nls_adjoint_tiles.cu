// nls_adjoint_tiles.cu -- root sensitivities (Sec. 2.3) for 8 < n <= 128.
//
// The same adjoint form as the thread kernel (nls_adjoint.cu): at a root u*
// with J = dF/du(u*), solve J^T mu = w for the cotangent w = dL/du* and
// return dL/dtheta = -mu^T dF/dtheta.  The Jacobian, the transpose and the
// solve reuse the solver tilings, in FP64:
//   * warp tiling (n <= 32): one instance per segment of L lanes; lane r
//     builds row r of J by forward-mode duals, the segment transposes it
//     through shared memory (lane r then holds row r of J^T) and runs the
//     solver's LU with partial pivoting on it;
//   * CTA tiling (n <= 128): one instance per 256-thread CTA; the R x R
//     register tiles of J are transposed through the CTA's shared-memory
//     factor buffer and factored by the solver's block-cyclic LU.
// Segments or CTAs without an instance of their own run on a copy of the
// last instance (every collective takes the full warp) and write nothing.
#include <algorithm>

#include <cuda_runtime.h>

#include "../../include/nls.h"
#include "nls_cta.cuh"
#include "nls_internal.h"
#include "nls_warp.cuh"

namespace nls {

struct AdjointTileArgs {
    const double *params; // [E][batch]
    const double *u;      // [n][batch] roots
    const double *w;      // [n][batch] dL/du
    double *grad;         // [E][batch] dL/dtheta
    int32_t *status;      // [batch] NLS_SUCCESS or NLS_SINGULAR (may be null)
    int64_t batch;
    int n;
};

// ---------------------------------------------------------------- warp

template <int L, int FAM>
__global__ void __launch_bounds__(WARP_TPB) k_adjoint_warp(AdjointTileArgs g)
{
    using S = WarpSolver<L, FAM, false>;
    using SM = WarpSmem<L, false>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int SEGS = 32 / L;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int seg = lane / L;
    SM &sm = reinterpret_cast<SM *>(smem_raw)[warp * SEGS + seg];
    const unsigned FULL = 0xffffffffu;
    const int64_t mine = ((int64_t)blockIdx.x * (WARP_TPB / 32) + warp) * SEGS + seg;
    const bool real = mine < g.batch;
    const int64_t k = real ? mine : g.batch - 1;
    const int64_t B = g.batch;

    S s;
    s.r = lane % L;
    s.n = g.n;
    s.lane0 = seg * L;
    SolveArgs a{};
    a.params = g.params;
    a.u = const_cast<double *>(g.u);
    a.batch = B;
    a.ld = B;
    a.n = g.n;
    a.maxiters = 1;
    s.init(a, k, sm, FULL); // parameters and the root; its residual is not used
    double row[L];
    s.jacobian_row(row);
    // transpose: lane r takes column r of J, i.e. row r of J^T
#pragma unroll
    for (int j = 0; j < L; ++j) sm.tr[s.r][j] = row[j];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < L; ++j) row[j] = sm.tr[j][s.r];
    __syncwarp();
    double mu = s.row_live() ? g.w[(int64_t)s.r * B + k] : 0.0;
    const bool ok = s.lu_solve(row, mu, sm); // mu_r = (J^-T w)_r in lane r
    const int n = g.n;
    if constexpr (FAM == FAM_CUBIC) {
        // dF_i/dA_ij = u_j, dF_i/db_i = -1; lane r writes row r of dL/dA
        sm.u[s.r] = s.u;
        __syncwarp();
        if (real && s.row_live()) {
            for (int j = 0; j < n; ++j) g.grad[(int64_t)(s.r * n + j) * B + k] = -mu * sm.u[j];
            g.grad[(int64_t)(n * n + s.r) * B + k] = mu;
        }
        __syncwarp();
    } else if constexpr (FAM == FAM_BRATU) {
        // dF_i/dlambda = exp(u_i)
        const double t = seg_sum<L>(s.row_live() ? mu * exp(s.u) : 0.0, FULL);
        if (real && s.r == 0) g.grad[k] = -t;
    } else if constexpr (FAM == FAM_SQUARE) {
        if (real && s.row_live()) g.grad[(int64_t)s.r * B + k] = mu;
    }
    if (real && s.r == 0 && g.status) g.status[k] = ok ? ST_SUCCESS : ST_SINGULAR;
}

template <int L, int FAM>
static cudaError_t launch_adjoint_warp_lf(const AdjointTileArgs &g, cudaStream_t st)
{
    constexpr int per_cta = (WARP_TPB / 32) * (32 / L);
    const int64_t grid = (g.batch + per_cta - 1) / per_cta;
    k_adjoint_warp<L, FAM><<<(unsigned)grid, WARP_TPB, warp_smem_bytes<L, false>(), st>>>(g);
    return cudaGetLastError();
}

template <int L>
static cudaError_t launch_adjoint_warp_l(int family, const AdjointTileArgs &g, cudaStream_t st)
{
    switch (family) {
    case FAM_CUBIC: return launch_adjoint_warp_lf<L, FAM_CUBIC>(g, st);
    case FAM_BRATU: return launch_adjoint_warp_lf<L, FAM_BRATU>(g, st);
    case FAM_SQUARE: return launch_adjoint_warp_lf<L, FAM_SQUARE>(g, st);
    case FAM_ROSENBROCK: return launch_adjoint_warp_lf<L, FAM_ROSENBROCK>(g, st);
    default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------- CTA

template <int R, int FAM>
__global__ void __launch_bounds__(CTA_TPB) k_adjoint_cta(AdjointTileArgs g)
{
    using S = CtaSolver<R, FAM, false>;
    using SM = typename S::SM;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SM &sm = *reinterpret_cast<SM *>(smem_raw);
    S s;
    s.tid = threadIdx.x;
    s.tx = s.tid / CTA_T;
    s.ty = s.tid % CTA_T;
    s.lane = s.tid & 31;
    s.warp = s.tid >> 5;
    s.n = g.n;
    s.B = g.batch;
    s.params = g.params;
    const int n = g.n;
    const int64_t B = g.batch;
    for (int64_t k = blockIdx.x; k < B; k += gridDim.x) {
        s.k = k;
        if (s.tid < n) sm.u[s.tid] = g.u[(int64_t)s.tid * B + k];
        if constexpr (FAM == FAM_BRATU) s.lam = __ldg(g.params + k);
        __syncthreads();
        double a[R][R];
        s.jacobian_tile(a, sm);
        // transpose through the factor buffer (the LU refills it at its end)
#pragma unroll
        for (int aa = 0; aa < R; ++aa)
#pragma unroll
            for (int bb = 0; bb < R; ++bb) sm.U[s.row(aa)][s.col(bb)] = a[aa][bb];
        __syncthreads();
#pragma unroll
        for (int aa = 0; aa < R; ++aa)
#pragma unroll
            for (int bb = 0; bb < R; ++bb) a[aa][bb] = sm.U[s.col(bb)][s.row(aa)];
        if (s.tid < n) sm.rhs[s.tid] = g.w[(int64_t)s.tid * B + k];
        __syncthreads();
        const bool ok = s.lu_solve(a, sm); // mu = J^-T w in sm.x
        if constexpr (FAM == FAM_CUBIC) {
            for (int idx = s.tid; idx < n * n; idx += CTA_TPB) {
                const int i = idx / n, j = idx - i * n;
                g.grad[(int64_t)idx * B + k] = -sm.x[i] * sm.u[j];
            }
            if (s.tid < n) g.grad[(int64_t)(n * n + s.tid) * B + k] = sm.x[s.tid];
        } else if constexpr (FAM == FAM_BRATU) {
            const double t = s.bsum(s.tid < n ? sm.x[s.tid] * exp(sm.u[s.tid]) : 0.0, sm);
            if (s.tid == 0) g.grad[k] = -t;
        } else if constexpr (FAM == FAM_SQUARE) {
            if (s.tid < n) g.grad[(int64_t)s.tid * B + k] = sm.x[s.tid];
        }
        if (s.tid == 0 && g.status) g.status[k] = ok ? ST_SUCCESS : ST_SINGULAR;
        __syncthreads();
    }
}

template <int R, int FAM>
static cudaError_t launch_adjoint_cta_rf(const AdjointTileArgs &g, cudaStream_t st)
{
    const int smem = cta_smem_bytes<false, R>();
    static const cudaError_t attr = cudaFuncSetAttribute(
        reinterpret_cast<const void *>(&k_adjoint_cta<R, FAM>), cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (attr != cudaSuccess) return attr;
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_adjoint_cta<R, FAM>, CTA_TPB, smem);
    const int64_t grid = std::min<int64_t>(g.batch, (int64_t)std::max(occ, 1) * sms);
    k_adjoint_cta<R, FAM><<<(unsigned)grid, CTA_TPB, smem, st>>>(g);
    return cudaGetLastError();
}

template <int R>
static cudaError_t launch_adjoint_cta_r(int family, const AdjointTileArgs &g, cudaStream_t st)
{
    switch (family) {
    case FAM_CUBIC: return launch_adjoint_cta_rf<R, FAM_CUBIC>(g, st);
    case FAM_BRATU: return launch_adjoint_cta_rf<R, FAM_BRATU>(g, st);
    case FAM_SQUARE: return launch_adjoint_cta_rf<R, FAM_SQUARE>(g, st);
    case FAM_ROSENBROCK: return launch_adjoint_cta_rf<R, FAM_ROSENBROCK>(g, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_adjoint_tiles(int family, int n, const double *params, const double *u, const double *w,
                                 double *grad, int32_t *status, int64_t batch, cudaStream_t st)
{
    AdjointTileArgs g{params, u, w, grad, status, batch, n};
    if (n <= 16) return launch_adjoint_warp_l<16>(family, g, st);
    if (n <= 32) return launch_adjoint_warp_l<32>(family, g, st);
    if (n <= 64) return launch_adjoint_cta_r<4>(family, g, st);
    if (n <= 128) return launch_adjoint_cta_r<8>(family, g, st);
    return cudaErrorInvalidValue;
}

} // namespace nls
