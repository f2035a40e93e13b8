// nls_cta_ext.cuh -- Potra-Ptak (Sec. 2.1, Eq. 4), Halley (Sec. 2.1, Eq. 3),
// Broyden and modified Broyden (Sec. 3.1, Tab. 1) on the CTA tiling: one
// instance per 256-thread CTA, 32 < n <= 128 (any n <= 16 R).
//
// The methods are those of the thread kernels (nls_thread_ext.cuh):
//  * Potra-Ptak and Halley factor J once per pass with the tiling's
//    block-cyclic LU, which leaves L \ U in position order in shared memory,
//    and solve the second right-hand side with CtaSolver::lu_apply.
//  * Halley's (H a a)_t comes from second-order jets over the stencil of
//    F_t, thread t owning component t.
//  * Broyden keeps B^-1 in the R x R register tiles that hold J in the
//    Newton kernels; products with vectors reduce the threads' partial sums
//    through shared memory (the tiling's J^T F pattern), and the rank-one
//    update touches each tile once.  Modified Broyden's start J(u_0)^-1 is
//    solved eight columns at a time, one unit vector per warp.
#pragma once

#include "nls_cta.cuh"
#include "nls_internal.h"

namespace nls {

template <int R, int FAM, bool MIXED>
struct CtaSolverExtBase : CtaSolver<R, FAM, MIXED> {
    using C = CtaSolver<R, FAM, MIXED>;
    using typename C::P;
    using typename C::SM;
    using C::tid;
    using C::tx;
    using C::ty;
    using C::n;
    using C::lam;
    using C::fF;
    using C::it;
    using C::nfev;
    using C::status;

    // (H a a)_t = d^2/dt^2 F_t(u + s a) at s = 0 by jets over the stencil of
    // F_t; u in sm.u, a in `dir` (both by component); t < n.
    NLS_DI P hvv_t(const SM &sm, const P *dir) const
    {
        const int t = tid;
        const P ut = P(sm.u[t]), at = dir[t];
        if constexpr (FAM == FAM_CUBIC) {
            const Jet<P, false> x{ut, at, P(0)};
            return (x * x * x).d2;
        } else if constexpr (FAM == FAM_BRATU) {
            const P inv_h2 = P((n + 1) * (n + 1));
            const Jet<P, false> xl{t > 0 ? P(sm.u[t - 1]) : P(0), t > 0 ? dir[t - 1] : P(0), P(0)};
            const Jet<P, false> xr{t < n - 1 ? P(sm.u[t + 1]) : P(0), t < n - 1 ? dir[t + 1] : P(0), P(0)};
            const Jet<P, false> xc{ut, at, P(0)};
            return (inv_h2 * ((xl + P(-2) * xc) + xr) + P(lam) * exp(xc)).d2;
        } else if constexpr (FAM == FAM_SQUARE) {
            const Jet<P, false> x{ut, at, P(0)};
            return (x * x).d2;
        } else {
            if (t == 0) return P(0);
            const Jet<P, false> xl{P(sm.u[t - 1]), dir[t - 1], P(0)}, xc{ut, at, P(0)};
            return (P(10) * (xc - xl * xl)).d2;
        }
    }

    // residual at sm.u into sm.F, norms and the convergence test (Sec. 2.1)
    NLS_DI void finish_pass(const SolveArgs &A, SM &sm)
    {
        const double f = this->residual_t(sm.u);
        ++nfev;
        __syncthreads();
        if (tid < n) sm.F[tid] = f;
        double f2 = f * f;
        uint64_t mx = mag_bits(f);
        this->bsum_max(f2, mx, sm);
        fF = f2;
        this->set_status_from(mx, A);
    }
};

// Potra-Ptak (ALG_POTRA_PTAK) and Halley (ALG_HALLEY).
template <int R, int FAM, bool MIXED, int ALG>
struct CtaSolverTwoSolve : CtaSolverExtBase<R, FAM, MIXED> {
    using Bx = CtaSolverExtBase<R, FAM, MIXED>;
    using typename Bx::P;
    using typename Bx::SM;
    using Bx::tid;
    using Bx::n;
    using Bx::it;
    using Bx::nfev;
    using Bx::status;

    NLS_DI void pass(const SolveArgs &A, SM &sm)
    {
        ++it;
        P a[R][R];
        this->jacobian_tile(a, sm);
        const int t = tid;
        const bool own = t < n;
        if (own) sm.rhs[t] = P(-sm.F[t]);
        __syncthreads();
        if (!this->lu_solve(a, sm)) { // the Newton step in sm.x, factors kept
            status = ST_SINGULAR;
            return;
        }
        if constexpr (ALG == ALG_POTRA_PTAK) {
            if (own) sm.ut[t] = sm.u[t] + double(sm.x[t]);
            __syncthreads();
            const double fy = this->residual_t(sm.ut);
            ++nfev;
            if (own) sm.rhs[t] = P(-fy);
            this->lu_apply(sm); // the same factors again
            if (own) sm.u[t] = sm.ut[t] + double(sm.x[t]);
        } else {
            const P at = own ? sm.x[t] : P(0);
            const P h = own ? this->hvv_t(sm, sm.x) : P(0);
            __syncthreads();
            if (own) sm.rhs[t] = h;
            this->lu_apply(sm); // J b = H a a
            if (own) {
                const P den = at + P(0.5) * sm.x[t];
                const P d = (den != P(0)) ? (at * at) / den : at;
                sm.u[t] += double(d);
            }
        }
        __syncthreads();
        this->finish_pass(A, sm);
    }
};

// Broyden (B_0 = I) and modified Broyden (B_0 = J(u_0)): H = B^-1 in the
// register tiles, Sherman-Morrison form of the good update.
template <int R, int FAM, bool MIXED>
struct CtaSolverBroyden : CtaSolverExtBase<R, FAM, MIXED> {
    using Bx = CtaSolverExtBase<R, FAM, MIXED>;
    using typename Bx::P;
    using typename Bx::SM;
    using Bx::tid;
    using Bx::tx;
    using Bx::ty;
    using Bx::n;
    using Bx::it;
    using Bx::nfev;
    using Bx::status;

    P H[R][R];
    bool need_start, singular_next;

    NLS_DI void init(const SolveArgs &A, SM &sm)
    {
        Bx::init(A, sm);
        need_start = true;
        singular_next = false;
    }

    // out = H v (rows) with v, out in shared memory by component
    NLS_DI void mv_rows(const P *v, P *out, SM &sm) const
    {
#pragma unroll
        for (int aa = 0; aa < R; ++aa) {
            P s = P(0);
#pragma unroll
            for (int bb = 0; bb < R; ++bb)
                if (this->col(bb) < n) s = fma(H[aa][bb], v[this->col(bb)], s);
            sm.red[tx][this->row(aa)] = s;
        }
        __syncthreads();
        if (tid < n) {
            P s = P(0);
#pragma unroll
            for (int q = 0; q < CTA_T; ++q) s += sm.red[q][tid];
            out[tid] = s;
        }
        __syncthreads();
    }

    // out = H^T v (columns)
    NLS_DI void mv_cols(const P *v, P *out, SM &sm) const
    {
#pragma unroll
        for (int bb = 0; bb < R; ++bb) {
            P s = P(0);
#pragma unroll
            for (int aa = 0; aa < R; ++aa)
                if (this->row(aa) < n) s = fma(H[aa][bb], v[this->row(aa)], s);
            sm.red[ty][this->col(bb)] = s;
        }
        __syncthreads();
        if (tid < n) {
            P s = P(0);
#pragma unroll
            for (int q = 0; q < CTA_T; ++q) s += sm.red[q][tid];
            out[tid] = s;
        }
        __syncthreads();
    }

    NLS_DI void pass(const SolveArgs &A, SM &sm)
    {
        ++it;
        if (singular_next) {
            status = ST_SINGULAR;
            return;
        }
        const int t = tid;
        const bool own = t < n;
        if (need_start) {
            need_start = false;
            if (A.alg == ALG_MOD_BROYDEN) {
                P a[R][R];
                this->jacobian_tile(a, sm);
                if (own) sm.rhs[t] = P(0);
                __syncthreads();
                // one factorisation per instance: the LU without row compaction
                // (which would only add registers here)
                if (!this->template lu_solve<false>(a, sm)) {
                    status = ST_SINGULAR;
                    return;
                }
#pragma unroll
                for (int aa = 0; aa < R; ++aa)
#pragma unroll
                    for (int bb = 0; bb < R; ++bb) H[aa][bb] = P(0);
                // J^-1 eight columns at a time: warp w solves for unit vector
                // j0 + w into row w of the partial-sum buffer, then the owners
                // of those columns copy them into their tiles
                constexpr int W = CTA_TPB / 32;
                for (int j0 = 0; j0 < n; j0 += W) {
                    const int j = j0 + this->warp;
                    if (j < n) {
                        P y[Bx::YJ];
#pragma unroll
                        for (int q = 0; q < Bx::YJ; ++q) {
                            const int p = this->lane + 32 * q;
                            y[q] = (p < n && sm.pos_row[p] == j) ? P(1) : P(0);
                        }
                        this->lu_apply_warp(sm, y, sm.red[this->warp]);
                    }
                    __syncthreads();
#pragma unroll
                    for (int aa = 0; aa < R; ++aa)
#pragma unroll
                        for (int bb = 0; bb < R; ++bb) {
                            const int c = this->col(bb);
                            if (c >= j0 && c < j0 + W && c < n && this->row(aa) < n)
                                H[aa][bb] = sm.red[c - j0][this->row(aa)];
                        }
                    __syncthreads();
                }
            } else {
#pragma unroll
                for (int aa = 0; aa < R; ++aa)
#pragma unroll
                    for (int bb = 0; bb < R; ++bb)
                        H[aa][bb] = (this->row(aa) == this->col(bb) && this->row(aa) < n) ? P(1) : P(0);
            }
        }
        // du = -H F
        if (own) sm.Fp[t] = P(sm.F[t]);
        __syncthreads();
        mv_rows(sm.Fp, sm.x, sm);
        const P d = own ? -sm.x[t] : P(0);
        if (own) sm.ut[t] = sm.u[t] + double(d);
        __syncthreads();
        const double f = this->residual_t(sm.ut);
        ++nfev;
        // H df and w = H^T du
        if (own) {
            sm.rhs[t] = P(f - sm.F[t]);
            sm.Fp[t] = d;
        }
        __syncthreads();
        mv_rows(sm.rhs, sm.g, sm);
        mv_cols(sm.Fp, sm.Jg, sm);
        const P hdf = own ? sm.g[t] : P(0);
        const P den = P(this->bsum(double(d * hdf), sm));
        const uint64_t dz = this->bmax(mag_bits(double(d)), sm);
        if (dz != 0) {
            if (den != P(0) && mag_bits(den) < inf_bits(den)) {
                if (own) sm.rhs[t] = (d - hdf) * rcp(den);
                __syncthreads();
#pragma unroll
                for (int aa = 0; aa < R; ++aa) {
                    if (this->row(aa) >= n) continue;
                    const P c = sm.rhs[this->row(aa)];
#pragma unroll
                    for (int bb = 0; bb < R; ++bb)
                        if (this->col(bb) < n) H[aa][bb] = fma(c, sm.Jg[this->col(bb)], H[aa][bb]);
                }
            } else {
                singular_next = true;
            }
        }
        if (own) {
            sm.u[t] = sm.ut[t];
            sm.F[t] = f;
        }
        __syncthreads();
        double f2 = f * f;
        uint64_t mx = mag_bits(f);
        this->bsum_max(f2, mx, sm);
        this->fF = f2;
        this->set_status_from(mx, A);
    }
};

template <int R, int FAM, bool MIXED, int ALG>
struct cta_ext_solver {
    using type = CtaSolverTwoSolve<R, FAM, MIXED, ALG>;
};
template <int R, int FAM, bool MIXED>
struct cta_ext_solver<R, FAM, MIXED, ALG_BROYDEN> {
    using type = CtaSolverBroyden<R, FAM, MIXED>;
};

template <int R, int FAM, bool MIXED, int ALG>
__global__ void __launch_bounds__(CTA_TPB) k_solve_cta_ext(SolveArgs a)
{
    cta_loop<typename cta_ext_solver<R, FAM, MIXED, ALG>::type>(a);
}

template <int R, int FAM, bool MIXED, int ALG>
cudaError_t launch_cta_ext(const SolveArgs &a, int grid, cudaStream_t st)
{
    k_solve_cta_ext<R, FAM, MIXED, ALG><<<grid, CTA_TPB, cta_smem_bytes<MIXED, R>(), st>>>(a);
    return cudaGetLastError();
}

template <int R, int FAM, bool MIXED, int ALG>
KernelInfo cta_ext_info()
{
    // more than 48 KB of dynamic shared memory needs an opt-in, once per kernel
    static const cudaError_t attr = cudaFuncSetAttribute(
        reinterpret_cast<const void *>(&k_solve_cta_ext<R, FAM, MIXED, ALG>),
        cudaFuncAttributeMaxDynamicSharedMemorySize, cta_smem_bytes<MIXED, R>());
    (void)attr;
    KernelInfo k;
    k.launch = &launch_cta_ext<R, FAM, MIXED, ALG>;
    k.func = reinterpret_cast<const void *>(&k_solve_cta_ext<R, FAM, MIXED, ALG>);
    k.block = CTA_TPB;
    k.smem = cta_smem_bytes<MIXED, R>();
    k.per_cta = 1;
    return k;
}

// ALG is ALG_POTRA_PTAK, ALG_HALLEY or ALG_BROYDEN (also serving
// ALG_MOD_BROYDEN); R = 4 for n <= 64, 8 for n <= 128.
template <int ALG, bool MIXED>
KernelInfo cta_ext_info_for(int family, int n)
{
    if (n <= 64) {
        switch (family) {
        case FAM_CUBIC: return cta_ext_info<4, FAM_CUBIC, MIXED, ALG>();
        case FAM_BRATU: return cta_ext_info<4, FAM_BRATU, MIXED, ALG>();
        case FAM_SQUARE: return cta_ext_info<4, FAM_SQUARE, MIXED, ALG>();
        case FAM_ROSENBROCK: return cta_ext_info<4, FAM_ROSENBROCK, MIXED, ALG>();
        default: return KernelInfo{};
        }
    }
    if (n <= 128) {
        switch (family) {
        case FAM_CUBIC: return cta_ext_info<8, FAM_CUBIC, MIXED, ALG>();
        case FAM_BRATU: return cta_ext_info<8, FAM_BRATU, MIXED, ALG>();
        case FAM_SQUARE: return cta_ext_info<8, FAM_SQUARE, MIXED, ALG>();
        case FAM_ROSENBROCK: return cta_ext_info<8, FAM_ROSENBROCK, MIXED, ALG>();
        default: return KernelInfo{};
        }
    }
    return KernelInfo{};
}

} // namespace nls
