// nls_thread_ext.cuh -- multi-step, higher-order and quasi-Newton solvers,
// one instance per GPU thread (n <= 8), on the lane loop of nls_thread.cuh.
//
//  * Potra-Ptak (Sec. 2.1, Eq. 4): the Jacobian J_k and its LU serve two
//    solves per pass, J_k du1 = -F(u_k), y = u_k + du1, J_k du2 = -F(y),
//    u_{k+1} = y + du2.  Two residuals per pass, one Jacobian.
//  * Halley (Sec. 2.1, Eq. 3): a = -J_k^-1 F(u_k), J_k b = H_k a a with
//    H_k a a the second directional derivative of F along a, taken by
//    forward mode on second-order jets (nls_dual.cuh), and the elementwise
//    step (a o a) / (a + b/2).  Where a_i + b_i/2 is exactly zero the step
//    component is a_i.
//  * Broyden and modified Broyden (Sec. 3.1, Tab. 1): no Jacobian after the
//    start.  The approximation B_k starts at the identity (Broyden) or at the
//    forward-mode Jacobian J(u_0) (modified Broyden) and takes the good
//    Broyden update B <- B + (df - B du) du^T / (du^T du) after every full
//    step.  The kernel keeps H = B^-1 instead and applies the same update in
//    its Sherman-Morrison form,
//        H <- H + (du - H df) (du^T H) / (du^T H df),
//    so a pass costs four n x n matrix-vector products and no
//    factorisation.  A zero step skips the update; du^T H df = 0 (the
//    updated B is singular) ends the instance SINGULAR at the next pass.
//    In FP64, H lives in shared memory, one column of N*N words per lane
//    after the staged parameters (element (i, j) of lane l at word
//    (i*N + j)*32 + l, so a warp's access touches 32 consecutive words):
//    held in registers next to u, F and the step it pushed the FP64 n = 8
//    kernel into local memory.  The FP32 H of mixed mode fits in registers.
//
// Precision: as in the Newton kernels, the residual, its norm test and the
// update of u are FP64; the Jacobian, jets, LU and B^-1 are FP64 or FP32
// (NLS_MIXED).
#pragma once

#include "nls_internal.h"
#include "nls_thread.cuh"

namespace nls {

template <int N, int FAM, bool MIXED>
struct ThreadSolverBase {
    using Core = ThreadSolver<N, FAM, MIXED, false>;
    using P = typename Core::P;
    using Fm = Family<FAM, N>;
    static constexpr int E = Fm::E;

    double u[N], F[N];
    int it, nfev, status;

    NLS_DI void init(const ParamView &pv, const SolveArgs &a, int64_t k)
    {
#pragma unroll
        for (int i = 0; i < N; ++i) u[i] = a.u[(int64_t)i * a.ld + k];
        Core::residual(pv, u, F);
        nfev = 1;
        it = 0;
        const uint64_t m = max_mag_bits(F);
        if (m >= INF64_BITS) status = ST_NONFINITE;
        else if (m <= mag_bits(a.abstol)) status = ST_SUCCESS;
        else if (a.maxiters <= 0) status = ST_MAXITERS;
        else status = ST_RUNNING;
    }

    NLS_DI void finish(const SolveArgs &a, int64_t k) const
    {
#pragma unroll
        for (int i = 0; i < N; ++i) a.u[(int64_t)i * a.ld + k] = u[i];
        if (a.status) a.status[k] = status;
        if (a.iters) a.iters[k] = it;
        if (a.resid) a.resid[k] = bits_to_double(max_mag_bits(F));
        if (a.nfev) a.nfev[k] = nfev;
        if (a.ngrad) a.ngrad[k] = 0;
    }

    // convergence test after a pass (Sec. 2.1)
    NLS_DI void test(const SolveArgs &a)
    {
        const uint64_t m = max_mag_bits(F);
        if (m >= INF64_BITS) status = ST_NONFINITE;
        else if (m <= mag_bits(a.abstol)) status = ST_SUCCESS;
        else if (it >= a.maxiters) status = ST_MAXITERS;
    }

    // (H a a)_i = d^2/dt^2 F_i(u + t a) at t = 0, by jets
    NLS_DI static void hvv(const ParamView &pv, const P (&up)[N], const P (&ap)[N], P (&h)[N])
    {
        static_for<0, N>([&](auto I) {
            constexpr int i = decltype(I)::value;
            h[i] = Fm::template row<i>(pv, JetVec<N, P>{up, ap}).d2;
        });
    }
};

// Potra-Ptak (ALG = ALG_POTRA_PTAK) and Halley (ALG = ALG_HALLEY).
template <int N, int FAM, bool MIXED, int ALG>
struct ThreadSolverTwoSolve : ThreadSolverBase<N, FAM, MIXED> {
    using B = ThreadSolverBase<N, FAM, MIXED>;
    using typename B::Core;
    using typename B::P;
    using B::u;
    using B::F;
    using B::it;
    using B::nfev;
    using B::status;

    NLS_DI void pass(const ParamView &pv, const SolveArgs &a)
    {
        ++it;
        P J[N][N], r[N], b[N];
        int piv[N];
        Core::jacobian(pv, u, J);
        if (!lu_factor<N, P>(J, piv, r)) {
            status = ST_SINGULAR;
            return;
        }
#pragma unroll
        for (int i = 0; i < N; ++i) b[i] = P(-F[i]);
        lu_apply<N, P>(J, piv, r, b); // b = a, the Newton step
        if constexpr (ALG == ALG_POTRA_PTAK) {
            double y[N];
#pragma unroll
            for (int i = 0; i < N; ++i) y[i] = u[i] + double(b[i]);
            Core::residual(pv, y, F);
            ++nfev;
#pragma unroll
            for (int i = 0; i < N; ++i) b[i] = P(-F[i]);
            lu_apply<N, P>(J, piv, r, b); // the same factors again
#pragma unroll
            for (int i = 0; i < N; ++i) u[i] = y[i] + double(b[i]);
        } else {
            P up[N], h[N];
#pragma unroll
            for (int i = 0; i < N; ++i) up[i] = P(u[i]);
            B::hvv(pv, up, b, h);
            lu_apply<N, P>(J, piv, r, h); // J b_halley = H a a
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const P den = b[i] + P(0.5) * h[i];
                const P d = (den != P(0)) ? (b[i] * b[i]) / den : b[i];
                u[i] += double(d);
            }
        }
        Core::residual(pv, u, F);
        ++nfev;
        B::test(a);
    }
};

// Broyden (identity start) and modified Broyden (J(u_0) start); the start is
// chosen by a.alg at the first pass.
template <int N, int FAM, bool MIXED>
struct ThreadSolverBroyden : ThreadSolverBase<N, FAM, MIXED> {
    using Bs = ThreadSolverBase<N, FAM, MIXED>;
    using typename Bs::Core;
    using typename Bs::P;
    using Bs::u;
    using Bs::F;
    using Bs::it;
    using Bs::nfev;
    using Bs::status;

    static constexpr bool H_SMEM = !MIXED;
    // shared memory per CTA: the staged parameters, then (FP64) H
    static constexpr int H_OFFSET = (thread_smem_bytes<N, FAM, MIXED>() + 15) / 16 * 16;
    static constexpr int SMEM = H_SMEM ? H_OFFSET + N * N * THREAD_TPB * (int)sizeof(P)
                                       : thread_smem_bytes<N, FAM, MIXED>();

    P *h;                          // FP64: this lane's B^-1, (i, j) at h[(i * N + j) * THREAD_TPB]
    P hr[H_SMEM ? 1 : N * N];      // FP32: B^-1 in registers
    bool singular_next;

    NLS_DI P &H(int i, int j)
    {
        if constexpr (H_SMEM) return h[(i * N + j) * THREAD_TPB];
        else return hr[i * N + j];
    }

    NLS_DI void init(const ParamView &pv, const SolveArgs &a, int64_t k)
    {
        extern __shared__ __align__(16) unsigned char smem_raw[];
        h = reinterpret_cast<P *>(smem_raw + H_OFFSET) + threadIdx.x;
        Bs::init(pv, a, k);
        singular_next = false;
    }

    NLS_DI void pass(const ParamView &pv, const SolveArgs &a)
    {
        ++it;
        if (singular_next) {
            status = ST_SINGULAR;
            return;
        }
        if (it == 1) {
            if (a.alg == ALG_MOD_BROYDEN) {
                // H = J(u_0)^-1, one column per unit vector
                P J[N][N], r[N];
                int piv[N];
                Core::jacobian(pv, u, J);
                if (!lu_factor<N, P>(J, piv, r)) {
                    status = ST_SINGULAR;
                    return;
                }
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    P e[N];
#pragma unroll
                    for (int i = 0; i < N; ++i) e[i] = (i == j) ? P(1) : P(0);
                    lu_apply<N, P>(J, piv, r, e);
#pragma unroll
                    for (int i = 0; i < N; ++i) H(i, j) = e[i];
                }
            } else {
#pragma unroll
                for (int i = 0; i < N; ++i)
#pragma unroll
                    for (int j = 0; j < N; ++j) H(i, j) = (i == j) ? P(1) : P(0);
            }
        }
        // du = -H F, full step
        P Fp[N], d[N];
#pragma unroll
        for (int i = 0; i < N; ++i) Fp[i] = P(F[i]);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            P s = P(0);
#pragma unroll
            for (int j = 0; j < N; ++j) s = fma(H(i, j), Fp[j], s);
            d[i] = -s;
        }
        double Fn[N];
#pragma unroll
        for (int i = 0; i < N; ++i) u[i] += double(d[i]);
        Core::residual(pv, u, Fn);
        ++nfev;
        // Sherman-Morrison form of the good Broyden update
        P df[N], Hdf[N], w[N];
#pragma unroll
        for (int i = 0; i < N; ++i) df[i] = P(Fn[i] - F[i]);
        P den = P(0);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            P s = P(0), t = P(0);
#pragma unroll
            for (int j = 0; j < N; ++j) {
                s = fma(H(i, j), df[j], s);
                t = fma(d[j], H(j, i), t);
            }
            Hdf[i] = s;
            w[i] = t; // (du^T H)_i
        }
#pragma unroll
        for (int i = 0; i < N; ++i) den = fma(d[i], Hdf[i], den);
        uint32_t dz = 0;
#pragma unroll
        for (int i = 0; i < N; ++i) dz |= (mag_bits(d[i]) != 0);
        if (dz) {
            if (den != P(0) && mag_bits(den) < inf_bits(den)) {
                const P rd = rcp(den);
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    const P c = (d[i] - Hdf[i]) * rd;
#pragma unroll
                    for (int j = 0; j < N; ++j) H(i, j) = fma(c, w[j], H(i, j));
                }
            } else {
                singular_next = true;
            }
        }
#pragma unroll
        for (int i = 0; i < N; ++i) F[i] = Fn[i];
        Bs::test(a);
    }
};

template <int N, int FAM, bool MIXED, int ALG>
struct ext_solver {
    using type = ThreadSolverTwoSolve<N, FAM, MIXED, ALG>;
};
template <int N, int FAM, bool MIXED>
struct ext_solver<N, FAM, MIXED, ALG_BROYDEN> {
    using type = ThreadSolverBroyden<N, FAM, MIXED>;
};

template <class S>
struct ext_smem {
    template <class T>
    static constexpr int get(decltype(T::SMEM) *) { return T::SMEM; }
    template <class T>
    static constexpr int get(...) { return -1; }
};

template <int N, int FAM, bool MIXED, int ALG>
constexpr int thread_ext_smem_bytes()
{
    using S = typename ext_solver<N, FAM, MIXED, ALG>::type;
    constexpr int extra = ext_smem<S>::template get<S>(nullptr);
    return extra >= 0 ? extra : thread_smem_bytes<N, FAM, MIXED>();
}

template <int N, int FAM, bool MIXED, int ALG>
__global__ void __launch_bounds__(THREAD_TPB) k_solve_thread_ext(SolveArgs a)
{
    thread_lanes<typename ext_solver<N, FAM, MIXED, ALG>::type, MIXED>(a);
}

template <int N, int FAM, bool MIXED, int ALG>
cudaError_t launch_thread_ext(const SolveArgs &a, int grid, cudaStream_t st)
{
    k_solve_thread_ext<N, FAM, MIXED, ALG><<<grid, THREAD_TPB, thread_ext_smem_bytes<N, FAM, MIXED, ALG>(), st>>>(a);
    return cudaGetLastError();
}

template <int N, int FAM, bool MIXED, int ALG>
KernelInfo thread_ext_info()
{
    KernelInfo k;
    k.launch = &launch_thread_ext<N, FAM, MIXED, ALG>;
    k.func = reinterpret_cast<const void *>(&k_solve_thread_ext<N, FAM, MIXED, ALG>);
    k.block = THREAD_TPB;
    k.smem = thread_ext_smem_bytes<N, FAM, MIXED, ALG>();
    k.per_cta = THREAD_TPB;
    return k;
}

template <int N, int FAM, int ALG>
KernelInfo thread_ext_info_n(bool mixed)
{
    return mixed ? thread_ext_info<N, FAM, true, ALG>() : thread_ext_info<N, FAM, false, ALG>();
}

// ALG is ALG_POTRA_PTAK, ALG_HALLEY or ALG_BROYDEN (which also serves
// ALG_MOD_BROYDEN).
template <int FAM, int ALG>
KernelInfo thread_ext_info_family(int n, bool mixed)
{
    switch (n) {
    case 1: return thread_ext_info_n<1, FAM, ALG>(mixed);
    case 2: return thread_ext_info_n<2, FAM, ALG>(mixed);
    case 3: return thread_ext_info_n<3, FAM, ALG>(mixed);
    case 4: return thread_ext_info_n<4, FAM, ALG>(mixed);
    case 5: return thread_ext_info_n<5, FAM, ALG>(mixed);
    case 6: return thread_ext_info_n<6, FAM, ALG>(mixed);
    case 7: return thread_ext_info_n<7, FAM, ALG>(mixed);
    case 8: return thread_ext_info_n<8, FAM, ALG>(mixed);
    default: return KernelInfo{};
    }
}

} // namespace nls
