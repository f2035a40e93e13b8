// nls_warp_ext.cuh -- Potra-Ptak (Sec. 2.1, Eq. 4), Halley (Sec. 2.1, Eq. 3),
// Broyden and modified Broyden (Sec. 3.1, Tab. 1) on the warp tiling: one
// instance per segment of L lanes, 8 < n <= L <= 32, lane r owning row r.
//
// The methods are those of the thread kernels (nls_thread_ext.cuh); what
// changes is the data layout:
//  * a factorisation that serves two solves: warp_lu_factor is the warp
//    LU with virtual pivoting (rows never move; each lane keeps the position
//    its row takes) that also stores each row's multiplier of step k in its
//    column k.  A row's final position is the step at which it was the
//    pivot, so warp_lu_apply can replay the elimination of any right-hand
//    side: at step k the lane at position k broadcasts its value and the
//    lanes at later positions subtract their stored multiple; the back
//    substitution is the solver's.
//  * Halley's (H a a)_r comes from second-order jets over the stencil of
//    F_r (the direction's neighbouring components by shuffles).
//  * Broyden keeps row r of B^-1 in lane r; the four products per pass use
//    the segment's shared-memory broadcast and transpose buffers.
// Every collective is taken by all lanes of the warp, segments that are idle
// or finished included (they compute on stale data and change nothing).
#pragma once

#include "nls_internal.h"
#include "nls_warp.cuh"

namespace nls {

// LU with partial pivoting of the segment's rows, kept for warp_lu_apply:
// on return lane r's row holds its multipliers in the columns before its
// final position `pos` and U from `pos` on; rc = 1 / pivot of row `pos`.
// Same pivot choice as WarpSolver::lu_solve.  Returns false (segment-
// uniform) on a zero or non-finite pivot.
template <int L, class P, class SM>
NLS_DI bool warp_lu_factor(P (&a)[L], int r, int n, SM &sm, int &pos, P &rc)
{
    using K = decltype(mag_bits(P(0)));
    const K inf = inf_bits(P(0));
    pos = r;
    const bool live = r < n;
    rc = P(0);
    bool ok = true;
#pragma unroll
    for (int k = 0; k < L; ++k) {
        if (k < n) {
            K m = mag_bits(a[k]);
            if (pos > k && m > inf) m = K(0);
            const bool cand = live && pos >= k;
            uint64_t key;
            if constexpr (sizeof(K) == 4) key = cand ? ((uint64_t)m << 32) | (uint32_t)(L - 1 - pos) : 0ull;
            else key = cand ? m : 0ull;
            uint64_t best = seg_max<L>(key, 0xffffffffu);
            int ppos;
            if constexpr (sizeof(K) == 4) {
                ppos = L - 1 - (int)(best & 0xffffffffu);
                best >>= 32;
            } else {
                const uint32_t tie = (cand && key == best) ? (uint32_t)(L - 1 - pos) : 0u;
                ppos = L - 1 - (int)seg_max<L>(tie, 0xffffffffu);
                if (best == 0) ppos = k;
            }
            const bool is_piv = cand && pos == ppos;
            if (best == 0 || best >= (uint64_t)inf) ok = false;
            if (is_piv) {
#pragma unroll
                for (int c = k; c < L; ++c) sm.prow[c] = a[c];
            }
            __syncwarp();
            const P pr = rcp(sm.prow[k]);
            if (cand && pos == k && !is_piv) pos = ppos;
            if (is_piv) {
                pos = k;
                rc = pr;
            }
            if (cand && !is_piv) {
                const P l = a[k] * pr;
#pragma unroll
                for (int c = k + 1; c < L; ++c) a[c] -= l * sm.prow[c];
                a[k] = l;
            }
            __syncwarp();
        }
    }
    return ok;
}

// b <- A^-1 b with the factors of warp_lu_factor (b: component r in lane r
// on entry and on return).
template <int L, class P, class SM>
NLS_DI void warp_lu_apply(const P (&a)[L], int r, int n, int pos, P rc, P &b, SM &sm)
{
    const bool live = r < n;
#pragma unroll
    for (int k = 0; k < L; ++k) {
        if (k < n) {
            if (live && pos == k) sm.prow[L] = b;
            __syncwarp();
            const P pb = sm.prow[L];
            __syncwarp();
            if (live && pos > k) b -= a[k] * pb;
        }
    }
    P x = P(0);
#pragma unroll
    for (int k = L - 1; k >= 0; --k) {
        if (k < n) {
            if (live && pos == k) sm.prow[0] = b * rc;
            __syncwarp();
            const P xk = sm.prow[0];
            __syncwarp();
            if (r == k) x = xk;
            if (live && pos < k) b -= a[k] * xk;
        }
    }
    b = x;
}

template <int L, int FAM, bool MIXED>
struct WarpSolverExtBase : WarpSolver<L, FAM, MIXED> {
    using W = WarpSolver<L, FAM, MIXED>;
    using typename W::P;
    using typename W::SM;
    using W::r;
    using W::n;
    using W::u;
    using W::F;
    using W::b_r;
    using W::fF;
    using W::fmag;
    using W::it;
    using W::nfev;
    using W::status;

    // (H a a)_r = d^2/dt^2 F_r(u + t a) at t = 0 by jets over the stencil of
    // F_r; ar is component r of a.  All lanes of the warp call it.
    NLS_DI P hvv_row(P ar) const
    {
        const unsigned FULL = 0xffffffffu;
        const P ur = P(u);
        P h = P(0);
        if constexpr (FAM == FAM_CUBIC) {
            const Jet<P, false> x{ur, ar, P(0)};
            h = (x * x * x).d2; // the linear part has no second derivative
        } else if constexpr (FAM == FAM_BRATU) {
            const P inv_h2 = P((n + 1) * (n + 1));
            P ul = __shfl_up_sync(FULL, ur, 1, L), al = __shfl_up_sync(FULL, ar, 1, L);
            P uR = __shfl_down_sync(FULL, ur, 1, L), aR = __shfl_down_sync(FULL, ar, 1, L);
            if (r == 0) ul = al = P(0);
            if (r >= n - 1) uR = aR = P(0);
            const Jet<P, false> xl{ul, al, P(0)}, xc{ur, ar, P(0)}, xr{uR, aR, P(0)};
            h = (inv_h2 * ((xl + P(-2) * xc) + xr) + P(b_r) * exp(xc)).d2;
        } else if constexpr (FAM == FAM_SQUARE) {
            const Jet<P, false> x{ur, ar, P(0)};
            h = (x * x).d2;
        } else {
            const P ul = __shfl_up_sync(FULL, ur, 1, L), al = __shfl_up_sync(FULL, ar, 1, L);
            const Jet<P, false> xl{ul, al, P(0)}, xc{ur, ar, P(0)};
            h = (r == 0) ? P(0) : (P(10) * (xc - xl * xl)).d2;
        }
        return this->row_live() ? h : P(0);
    }

    // norms and the convergence test after a pass (Sec. 2.1)
    NLS_DI void test(const SolveArgs &A, bool run, bool go)
    {
        const unsigned FULL = 0xffffffffu;
        const double f2 = seg_sum<L>(F * F, FULL);
        const uint64_t m = seg_max<L>(mag_bits(F), FULL);
        if (run) {
            fF = f2;
            fmag = m;
        }
        if (go) {
            if (m >= INF64_BITS) status = ST_NONFINITE;
            else if (m <= mag_bits(A.abstol)) status = ST_SUCCESS;
            else if (it >= A.maxiters) status = ST_MAXITERS;
        }
    }
};

// Potra-Ptak (ALG_POTRA_PTAK) and Halley (ALG_HALLEY).
template <int L, int FAM, bool MIXED, int ALG>
struct WarpSolverTwoSolve : WarpSolverExtBase<L, FAM, MIXED> {
    using Bx = WarpSolverExtBase<L, FAM, MIXED>;
    using typename Bx::P;
    using typename Bx::SM;
    using Bx::r;
    using Bx::n;
    using Bx::u;
    using Bx::F;
    using Bx::it;
    using Bx::nfev;
    using Bx::status;

    NLS_DI void pass(const SolveArgs &A, SM &sm, bool run)
    {
        const unsigned FULL = 0xffffffffu;
        if (run) ++it;
        P a[L];
        this->jacobian_row(a);
        int pos;
        P rc;
        const bool ok = warp_lu_factor<L>(a, r, n, sm, pos, rc);
        if (run && !ok) status = ST_SINGULAR;
        const bool go = run && ok;
        P b = this->row_live() ? P(-F) : P(0);
        warp_lu_apply<L>(a, r, n, pos, rc, b, sm); // the Newton step, component r
        double un, Fn;
        if constexpr (ALG == ALG_POTRA_PTAK) {
            const double y = this->row_live() ? u + double(b) : 0.0;
            const double Fy = this->residual(y, sm, FULL);
            P b2 = P(-Fy);
            warp_lu_apply<L>(a, r, n, pos, rc, b2, sm); // the same factors again
            un = this->row_live() ? y + double(b2) : 0.0;
            Fn = this->residual(un, sm, FULL);
            if (go) nfev += 2;
        } else {
            P h = this->hvv_row(b);
            warp_lu_apply<L>(a, r, n, pos, rc, h, sm); // J b_halley = H a a
            const P den = b + P(0.5) * h;
            const P d = (den != P(0)) ? (b * b) / den : b;
            un = this->row_live() ? u + double(d) : 0.0;
            Fn = this->residual(un, sm, FULL);
            if (go) nfev += 1;
        }
        if (go) {
            u = un;
            F = Fn;
        }
        this->test(A, run, go);
    }
};

// Broyden (B_0 = I) and modified Broyden (B_0 = J(u_0)); lane r keeps row r
// of H = B^-1 and applies the Sherman-Morrison form of the good update.
template <int L, int FAM, bool MIXED>
struct WarpSolverBroyden : WarpSolverExtBase<L, FAM, MIXED> {
    using Bx = WarpSolverExtBase<L, FAM, MIXED>;
    using typename Bx::P;
    using typename Bx::SM;
    using Bx::r;
    using Bx::n;
    using Bx::u;
    using Bx::F;
    using Bx::it;
    using Bx::nfev;
    using Bx::status;

    P Hr[L];
    bool need_start, singular_next;

    NLS_DI void init(const SolveArgs &A, int64_t k, SM &sm, unsigned mask)
    {
        Bx::init(A, k, sm, mask);
        need_start = true;
        singular_next = false;
    }

    NLS_DI void pass(const SolveArgs &A, SM &sm, bool run)
    {
        const unsigned FULL = 0xffffffffu;
        if (run) ++it;
        bool failed = false;
        if (run && singular_next) {
            status = ST_SINGULAR;
            failed = true;
        }
        if (__any_sync(FULL, run && need_start)) {
            const bool fresh = run && need_start && !failed;
            if (A.alg == ALG_MOD_BROYDEN) {
                // H = J(u_0)^-1, one column per unit vector
                P a[L];
                this->jacobian_row(a);
                int pos;
                P rc;
                const bool ok = warp_lu_factor<L>(a, r, n, sm, pos, rc);
                // column j of J^-1 lands in lane r's own row r of the transpose
                // buffer (a runtime loop: the solve is emitted once)
#pragma unroll 1
                for (int j = 0; j < n; ++j) {
                    P e = (r == j && this->row_live()) ? P(1) : P(0);
                    warp_lu_apply<L>(a, r, n, pos, rc, e, sm);
                    sm.tr[r][j] = e;
                }
                __syncwarp();
                if (fresh) {
#pragma unroll
                    for (int j = 0; j < L; ++j) Hr[j] = (j < n) ? sm.tr[r][j] : P(0);
                }
                __syncwarp();
                if (fresh && !ok) {
                    status = ST_SINGULAR;
                    failed = true;
                }
            } else if (fresh) {
#pragma unroll
                for (int j = 0; j < L; ++j) Hr[j] = (j == r && this->row_live()) ? P(1) : P(0);
            }
            if (fresh) need_start = false;
        }
        const bool go = run && !failed;
        // du = -H F
        sm.vec[r] = P(F);
        __syncwarp();
        P d = P(0);
#pragma unroll
        for (int j = 0; j < L; ++j) d = fma(Hr[j], sm.vec[j], d);
        d = this->row_live() ? -d : P(0);
        __syncwarp();
        const double un = this->row_live() ? u + double(d) : 0.0;
        const double Fn = this->residual(un, sm, FULL);
        // H df and w = H^T du
        sm.vec[r] = P(Fn - F);
        __syncwarp();
        P Hdf = P(0);
#pragma unroll
        for (int j = 0; j < L; ++j) Hdf = fma(Hr[j], sm.vec[j], Hdf);
        __syncwarp();
#pragma unroll
        for (int j = 0; j < L; ++j) sm.tr[r][j] = d * Hr[j];
        __syncwarp();
        P w = P(0);
#pragma unroll
        for (int i = 0; i < L; ++i) w += sm.tr[i][r];
        __syncwarp();
        sm.vec[r] = w;
        __syncwarp();
        const P den = seg_sum<L>(d * Hdf, FULL);
        const bool dz = seg_max<L>(mag_bits(d), FULL) != 0;
        if (go && dz) {
            if (den != P(0) && mag_bits(den) < inf_bits(den)) {
                const P c = (d - Hdf) * rcp(den);
#pragma unroll
                for (int j = 0; j < L; ++j) Hr[j] = fma(c, sm.vec[j], Hr[j]);
            } else {
                singular_next = true;
            }
        }
        __syncwarp();
        if (go) {
            u = un;
            F = Fn;
            nfev += 1;
        }
        this->test(A, run, go);
    }
};

template <int L, int FAM, bool MIXED, int ALG>
struct warp_ext_solver {
    using type = WarpSolverTwoSolve<L, FAM, MIXED, ALG>;
};
template <int L, int FAM, bool MIXED>
struct warp_ext_solver<L, FAM, MIXED, ALG_BROYDEN> {
    using type = WarpSolverBroyden<L, FAM, MIXED>;
};

template <int L, int FAM, bool MIXED, int ALG>
__global__ void __launch_bounds__(WARP_TPB) k_solve_warp_ext(SolveArgs a)
{
    warp_lanes<typename warp_ext_solver<L, FAM, MIXED, ALG>::type, L, MIXED>(a);
}

template <int L, int FAM, bool MIXED, int ALG>
cudaError_t launch_warp_ext(const SolveArgs &a, int grid, cudaStream_t st)
{
    k_solve_warp_ext<L, FAM, MIXED, ALG><<<grid, WARP_TPB, warp_smem_bytes<L, MIXED>(), st>>>(a);
    return cudaGetLastError();
}

template <int L, int FAM, bool MIXED, int ALG>
KernelInfo warp_ext_info()
{
    KernelInfo k;
    k.launch = &launch_warp_ext<L, FAM, MIXED, ALG>;
    k.func = reinterpret_cast<const void *>(&k_solve_warp_ext<L, FAM, MIXED, ALG>);
    k.block = WARP_TPB;
    k.smem = warp_smem_bytes<L, MIXED>();
    k.per_cta = (WARP_TPB / 32) * (32 / L);
    return k;
}

// ALG is ALG_POTRA_PTAK, ALG_HALLEY or ALG_BROYDEN (also serving
// ALG_MOD_BROYDEN); L = 16 or 32.
template <int ALG, bool MIXED>
KernelInfo warp_ext_info_for(int family, int L)
{
    if (L == 16) {
        switch (family) {
        case FAM_CUBIC: return warp_ext_info<16, FAM_CUBIC, MIXED, ALG>();
        case FAM_BRATU: return warp_ext_info<16, FAM_BRATU, MIXED, ALG>();
        case FAM_SQUARE: return warp_ext_info<16, FAM_SQUARE, MIXED, ALG>();
        case FAM_ROSENBROCK: return warp_ext_info<16, FAM_ROSENBROCK, MIXED, ALG>();
        default: return KernelInfo{};
        }
    }
    if (L == 32) {
        switch (family) {
        case FAM_CUBIC: return warp_ext_info<32, FAM_CUBIC, MIXED, ALG>();
        case FAM_BRATU: return warp_ext_info<32, FAM_BRATU, MIXED, ALG>();
        case FAM_SQUARE: return warp_ext_info<32, FAM_SQUARE, MIXED, ALG>();
        case FAM_ROSENBROCK: return warp_ext_info<32, FAM_ROSENBROCK, MIXED, ALG>();
        default: return KernelInfo{};
        }
    }
    return KernelInfo{};
}

} // namespace nls
