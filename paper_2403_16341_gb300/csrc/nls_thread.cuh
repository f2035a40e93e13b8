// nls_thread.cuh -- one instance per GPU thread, for n <= 8 (compile-time N).
//
// The paper's GPU path (Sec. 3.3) runs one statically sized, non-allocating
// solver per GPU thread.  Here each lane of a warp owns an instance slot and
// keeps its state in registers: u and F in FP64, the Jacobian and its LU in
// FP64 or (NLS_MIXED) FP32.  Parameters are staged once per instance into the
// lane's own shared-memory column (no block synchronisation is needed).
//
// One loop pass per instance is one Newton iteration (Sec. 2.1, Eq. 2): the
// Jacobian by forward-mode duals (Sec. 2.4) or the analytic formula, LU with
// partial pivoting (Sec. 3.2), then the step of the chosen globalisation:
// full step, backtracking on the Armijo condition (Sec. 2.2.1, Eq. 8-9), or
// the dogleg trust-region step with the ratio test (Sec. 2.2.2, Eq. 13-15).
// Convergence is ||F||_inf <= abstol (Sec. 2.1).
//
// Scheduling: all lanes of a warp execute the same pass in lock step (a
// per-lane running mask), and in a persistent launch a warp refills its idle
// lanes from a global work counter whenever the number of running lanes
// drops to `refill_below` -- the lanes that finished early are given new
// instances instead of idling until the slowest lane of the warp finishes.
#pragma once

#include "nls_common.cuh"

namespace nls {

// ---------------------------------------------------------------------------
// Dense LU with partial pivoting on a register matrix, fused with the
// elimination of the right-hand side.  Row swaps are selects over the
// compile-time rows (a dynamic row index would force the matrix into local
// memory).  Pivot: first index of the largest |a_ik|, i >= k, comparing
// IEEE bit patterns; a NaN below the diagonal is never chosen and a NaN on
// the diagonal is kept (the same choices as the comparison |a_ik| > best).
// On return b holds x = A^-1 b.  Returns false on a zero / non-finite pivot.
template <int N, class P>
NLS_DI bool lu_solve(P (&a)[N][N], P (&b)[N])
{
    using K = decltype(mag_bits(P(0)));
    const K inf = inf_bits(P(0));
    P r[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
        K best = mag_bits(a[k][k]);
        int p = k;
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            K m = mag_bits(a[i][k]);
            m = (m > inf) ? K(0) : m;
            if (m > best) { best = m; p = i; }
        }
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            const bool s = (p == i);
#pragma unroll
            for (int j = k; j < N; ++j) {
                P t = a[k][j];
                a[k][j] = s ? a[i][j] : t;
                a[i][j] = s ? t : a[i][j];
            }
            P t = b[k];
            b[k] = s ? b[i] : t;
            b[i] = s ? t : b[i];
        }
        const K pm = mag_bits(a[k][k]);
        if (pm == K(0) || pm >= inf) return false;
        r[k] = rcp(a[k][k]);
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            const P l = a[i][k] * r[k];
#pragma unroll
            for (int j = k + 1; j < N; ++j) a[i][j] -= l * a[k][j];
            b[i] -= l * b[k];
        }
    }
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
        P s = b[i];
#pragma unroll
        for (int j = i + 1; j < N; ++j) s -= a[i][j] * b[j];
        b[i] = s * r[i];
    }
    return true;
}

// LU with partial pivoting that keeps its factors for later solves: on
// return a holds U on and above the diagonal and the multipliers of L below
// it, piv[k] is the row exchanged with row k at step k (whole rows move, so
// the stored multipliers follow their rows) and r[k] = 1 / u_kk.  Same pivot
// choice as lu_solve.  Returns false on a zero / non-finite pivot.
template <int N, class P>
NLS_DI bool lu_factor(P (&a)[N][N], int (&piv)[N], P (&r)[N])
{
    using K = decltype(mag_bits(P(0)));
    const K inf = inf_bits(P(0));
#pragma unroll
    for (int k = 0; k < N; ++k) {
        K best = mag_bits(a[k][k]);
        int p = k;
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            K m = mag_bits(a[i][k]);
            m = (m > inf) ? K(0) : m;
            if (m > best) { best = m; p = i; }
        }
        piv[k] = p;
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            const bool s = (p == i);
#pragma unroll
            for (int j = 0; j < N; ++j) {
                P t = a[k][j];
                a[k][j] = s ? a[i][j] : t;
                a[i][j] = s ? t : a[i][j];
            }
        }
        const K pm = mag_bits(a[k][k]);
        if (pm == K(0) || pm >= inf) return false;
        r[k] = rcp(a[k][k]);
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            const P l = a[i][k] * r[k];
            a[i][k] = l;
#pragma unroll
            for (int j = k + 1; j < N; ++j) a[i][j] -= l * a[k][j];
        }
    }
    return true;
}

// b <- A^-1 b from the factors of lu_factor: the row exchanges in order,
// then L y = P b (unit diagonal) and U x = y.
template <int N, class P>
NLS_DI void lu_apply(const P (&a)[N][N], const int (&piv)[N], const P (&r)[N], P (&b)[N])
{
#pragma unroll
    for (int k = 0; k < N; ++k) {
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            const bool s = (piv[k] == i);
            P t = b[k];
            b[k] = s ? b[i] : t;
            b[i] = s ? t : b[i];
        }
    }
#pragma unroll
    for (int k = 0; k < N; ++k)
#pragma unroll
        for (int i = k + 1; i < N; ++i) b[i] -= a[i][k] * b[k];
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
        P s = b[i];
#pragma unroll
        for (int j = i + 1; j < N; ++j) s -= a[i][j] * b[j];
        b[i] = s * r[i];
    }
}

template <class R>
struct mask_of;
template <int M_N, uint32_t M, class T>
struct mask_of<Dual<M_N, M, T>> {
    static constexpr uint32_t value = M;
};

constexpr int THREAD_TPB = 32; // one warp per CTA: lanes never wait on each other

template <int N, int FAM, bool MIXED>
constexpr int thread_smem_bytes()
{
    return THREAD_TPB * family_params<FAM>(N) * (8 + (MIXED ? 4 : 0));
}

// The FP64 Newton-family kernel also keeps the trust region's g = J^T F and
// J g in the lane's shared-memory columns, after the staged parameters (in
// mixed precision they are FP32 and stay in registers: their shared copy
// would cost an eighth CTA per SM).
template <int N, int FAM, bool MIXED>
constexpr int thread_newton_smem_bytes()
{
    return MIXED ? thread_smem_bytes<N, FAM, MIXED>()
                 : (thread_smem_bytes<N, FAM, MIXED>() + 15) / 16 * 16 + 2 * N * THREAD_TPB * 8;
}

template <int N, int FAM, bool MIXED, bool ANALYTIC>
struct ThreadSolver {
    using P = typename std::conditional<MIXED, float, double>::type;
    using Fm = Family<FAM, N>;
    static constexpr int E = Fm::E;

    // F(u) in FP64 (all families, all modes)
    NLS_DI static void residual(const ParamView &pv, const double (&u)[N], double (&F)[N])
    {
        static_for<0, N>([&](auto I) {
            constexpr int i = decltype(I)::value;
            F[i] = Fm::template row<i>(pv, PlainVec<N, double>{u});
        });
    }

    // J(u) in the Jacobian precision P
    NLS_DI static void jacobian(const ParamView &pv, const double (&u)[N], P (&J)[N][N])
    {
        P up[N];
#pragma unroll
        for (int i = 0; i < N; ++i) up[i] = P(u[i]);
        if constexpr (ANALYTIC) {
            Fm::template jac_analytic<P>(pv, up, J);
        } else {
            static_for<0, N>([&](auto I) {
                constexpr int i = decltype(I)::value;
                const auto r = Fm::template row<i>(pv, SeedVec<N, P>{up});
                using R = typename std::decay<decltype(r)>::type;
                static_for<0, N>([&](auto Jc) {
                    constexpr int j = decltype(Jc)::value;
                    J[i][j] = dual_has<R>(j) ? r.d[j] : P(0);
                });
            });
        }
    }

    template <class R>
    NLS_DI static constexpr bool dual_has(int j) { return (mask_of<R>::value >> j) & 1u; }

    NLS_DI static double sumsq(const double (&v)[N])
    {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < N; ++i) s = fma(v[i], v[i], s);
        return s;
    }

    // ------------------------------------------------------------ lane state
    double u[N], F[N], dN[N];
    // g = J^T F and J g of the trust region.  FP64: element j of the lane's
    // column in shared memory (out of the register file, which J, u, F and
    // the Newton step fill); mixed: FP32 registers.
    P greg_[MIXED ? N : 1], jgreg_[MIXED ? N : 1];
    NLS_DI static P *gcol()
    {
        extern __shared__ __align__(16) unsigned char smem_raw[];
        constexpr int off = (thread_smem_bytes<N, FAM, MIXED>() + 15) / 16 * 16;
        return reinterpret_cast<P *>(smem_raw + off) + threadIdx.x;
    }
    NLS_DI P &g(int j)
    {
        if constexpr (MIXED) return greg_[j];
        else return gcol()[j * THREAD_TPB];
    }
    NLS_DI P &Jg(int i)
    {
        if constexpr (MIXED) return jgreg_[i];
        else return gcol()[(N + i) * THREAD_TPB];
    }
    // F and the Newton step in the Jacobian precision; in FP64 mode they are
    // F and dN themselves (no second copy across passes)
    P Fp_[MIXED ? N : 1], dNp_[MIXED ? N : 1];
    NLS_DI P Fp(int i) const
    {
        if constexpr (MIXED) return Fp_[i];
        else return F[i];
    }
    NLS_DI P dNp(int i) const
    {
        if constexpr (MIXED) return dNp_[i];
        else return dN[i];
    }
    double fF, Delta;
    int it, nfev, rej, status;
    int ngrad;   // trust region: passes that formed g and J g
    bool need_jac;
    bool have_g; // trust region: g = J^T F and J g formed for the current J

    NLS_DI void init(const ParamView &pv, const SolveArgs &a, int64_t k)
    {
#pragma unroll
        for (int i = 0; i < N; ++i) u[i] = a.u[(int64_t)i * a.ld + k];
        residual(pv, u, F);
        nfev = 1;
        it = 0;
        rej = 0;
        ngrad = 0;
        Delta = TR_DELTA0;
        need_jac = true;
        have_g = false;
        fF = sumsq(F);
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
        if (a.ngrad) a.ngrad[k] = ngrad;
    }

    // g = J^T Fp and, with jg, J g.
    NLS_DI void gradient(const P (&J)[N][N], bool jg)
    {
#pragma unroll
        for (int j = 0; j < N; ++j) {
            P s = P(0);
#pragma unroll
            for (int i = 0; i < N; ++i) s = fma(J[i][j], Fp(i), s);
            g(j) = s;
        }
        if (jg) {
#pragma unroll
            for (int i = 0; i < N; ++i) {
                P s = P(0);
#pragma unroll
                for (int j = 0; j < N; ++j) s = fma(J[i][j], g(j), s);
                Jg(i) = s;
            }
        }
    }

    // One loop pass (Jacobian use) of the chosen algorithm.
    NLS_DI void pass(const ParamView &pv, const SolveArgs &a)
    {
        ++it;
        if (need_jac) {
            P J[N][N], b[N];
            jacobian(pv, u, J);
#pragma unroll
            for (int i = 0; i < N; ++i)
                if constexpr (MIXED) Fp_[i] = P(F[i]);
            // the trust region forms g = J^T F and J g only when the Newton step
            // leaves the region (J is re-evaluated then: the LU overwrites it)
            have_g = false;
#pragma unroll
            for (int i = 0; i < N; ++i) b[i] = -Fp(i);
            if (!lu_solve<N, P>(J, b)) {
                status = ST_SINGULAR;
                return;
            }
#pragma unroll
            for (int i = 0; i < N; ++i) {
                if constexpr (MIXED) dNp_[i] = b[i];
                dN[i] = double(b[i]);
            }
            need_jac = false;
        }

        if (a.alg == ALG_NEWTON) {
#pragma unroll
            for (int i = 0; i < N; ++i) u[i] += dN[i];
            residual(pv, u, F);
            ++nfev;
            need_jac = true;
        } else if (a.alg == ALG_NEWTON_BACKTRACK) {
            // slope F^T J dN of Eq. 9 by linearity: J dN = -F, so it is -||F||^2
            // (no J^T F is formed); phi(alpha) = 1/2 ||F(u + alpha dN)||^2
            const double s = -fF;
            const double phi0 = 0.5 * fF;
            double alpha = 1.0;
            bool ok = false;
            for (int m = 0; m < LS_MAX_TRIALS; ++m) {
                double ut[N], Ft[N];
#pragma unroll
                for (int i = 0; i < N; ++i) ut[i] = fma(alpha, dN[i], u[i]);
                residual(pv, ut, Ft);
                ++nfev;
                const double fFt = sumsq(Ft);
                if (max_mag_bits(Ft) < INF64_BITS && 0.5 * fFt <= phi0 + LS_C1 * alpha * s) {
#pragma unroll
                    for (int i = 0; i < N; ++i) { u[i] = ut[i]; F[i] = Ft[i]; }
                    fF = fFt;
                    ok = true;
                    break;
                }
                alpha *= LS_RHO;
            }
            if (!ok) {
                status = ST_LS_FAILED;
                return;
            }
            need_jac = true;
        } else {
            // Powell's dogleg on m(d) = 1/2||F||^2 + d^T J^T F + 1/2 d^T J^T J d, ||d||_2 <= Delta.
            // pred = ||F||^2 - ||F + J d||^2 = -2 F.Jd - ||Jd||^2 (Eq. 15) by linearity:
            // J dN = -F and, with g = J^T F, F.(J g) = g.g, so every branch's pred is
            // a combination of ||F||^2, ||g||^2 and ||J g||^2 (no vector J d is formed).
            double d[N];
            double pred;
            const P D2 = P(Delta * Delta);
            P nN2 = P(0);
#pragma unroll
            for (int i = 0; i < N; ++i) nN2 = fma(dNp(i), dNp(i), nN2);
            const bool boundary = !(nN2 <= D2);
            if (nN2 <= D2) {
#pragma unroll
                for (int i = 0; i < N; ++i) d[i] = dN[i];
                pred = fF; // J dN = -F
            } else {
                if (!have_g) {
                    // J at the same u again (the LU overwrote it): same values as before
                    P J[N][N];
                    jacobian(pv, u, J);
                    gradient(J, true);
                    have_g = true;
                    ++ngrad;
                }
                P gg = P(0), JgJg = P(0);
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    const P gi = g(i), jgi = Jg(i);
                    gg = fma(gi, gi, gg);
                    JgJg = fma(jgi, jgi, JgJg);
                }
                const P t = gg / JgJg; // Cauchy point c = -t g minimises m along -g
                const P cc = t * t * gg;
                if (cc >= D2) {
                    const P sc = P(Delta) / nls_sqrt(gg);
#pragma unroll
                    for (int i = 0; i < N; ++i) d[i] = double(-sc * g(i));
                    pred = double(sc * (P(2) * gg - sc * JgJg)); // J d = -sc J g
                } else {
                    P w[N], aa = P(0), bb = P(0);
#pragma unroll
                    for (int i = 0; i < N; ++i) {
                        const P gi = g(i);
                        w[i] = dNp(i) + t * gi;
                        aa = fma(w[i], w[i], aa);
                        bb = fma(-t * gi, w[i], bb);
                    }
                    const P q = cc - D2;
                    const P tau = (-bb + nls_sqrt(bb * bb - aa * q)) / aa;
#pragma unroll
                    for (int i = 0; i < N; ++i) d[i] = double(fma(tau, w[i], -t * g(i)));
                    // J d = -s1 J g - tau F with s1 = (1 - tau) t
                    const P s1 = (P(1) - tau) * t;
                    pred = double(s1 * (P(2) * (P(1) - tau) * gg - s1 * JgJg) + tau * (P(2) - tau) * P(fF));
                }
            }
            double ut[N], Ft[N];
#pragma unroll
            for (int i = 0; i < N; ++i) ut[i] = u[i] + d[i];
            residual(pv, ut, Ft);
            ++nfev;
            const double fFt = sumsq(Ft);
            // rho = ared / pred (Eq. 15)
            const double ared = fF - fFt;
            const bool ok = pred > 0.0 && max_mag_bits(Ft) < INF64_BITS;
            if (tr_step_outcome(a.tr_scheme, ok, ared, pred, boundary, Delta)) {
#pragma unroll
                for (int i = 0; i < N; ++i) { u[i] = ut[i]; F[i] = Ft[i]; }
                fF = fFt;
                need_jac = true;
                rej = 0;
            } else {
                if (++rej >= TR_MAX_REJECTIONS) {
                    status = ST_TR_STALLED;
                    return;
                }
            }
        }
        const uint64_t m = max_mag_bits(F);
        if (m >= INF64_BITS) status = ST_NONFINITE;
        else if (m <= mag_bits(a.abstol)) status = ST_SUCCESS;
        else if (it >= a.maxiters) status = ST_MAXITERS;
    }
};

// The lane loop shared by every one-instance-per-thread solver S (S::E
// parameters, init / pass / finish, a status): each lane owns an instance
// slot, all lanes of the warp step in lock step, and idle lanes are refilled
// from the work counter (persistent launches) or from the static slot.
template <class S, bool MIXED>
NLS_DI void thread_lanes(SolveArgs &a)
{
    apply_dyn_batch(a);
    constexpr int E = S::E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *sd = reinterpret_cast<double *>(smem_raw);
    float *sf = reinterpret_cast<float *>(sd + E * THREAD_TPB);
    const int lane = threadIdx.x;
    const ParamView pv{sd + lane, sf + lane, THREAD_TPB};
    const unsigned FULL = 0xffffffffu;

    const unsigned long long t_end = a.budget_ns ? global_ns() + a.budget_ns : ~0ull;
    S s;
    bool have = false;     // lane holds a running instance
    bool exhausted = false; // no more work for this warp
    int64_t k = -1;
    bool first = true;
    unsigned long long local_solved = 0;

    for (;;) {
        const int live = __popc(__ballot_sync(FULL, have));
        if (!exhausted && live <= a.refill_below) {
            const bool want = !have;
            int64_t cand = a.batch;
            if (a.counter == nullptr) {
                if (first && want) cand = (int64_t)blockIdx.x * THREAD_TPB + lane;
            } else {
                const unsigned m = __ballot_sync(FULL, want);
                if (want) {
                    const int leader = __ffs(m) - 1;
                    unsigned long long base = 0;
                    if (lane == leader) base = atomicAdd(a.counter, (unsigned long long)__popc(m));
                    base = __shfl_sync(m, base, leader);
                    cand = (int64_t)base + __popc(m & ((1u << lane) - 1u));
                }
            }
            first = false;
            bool got = false;
            // A whole warp taking 32 consecutive instances whose first is even
            // (every full refill and every static slot; ld even, params 16-byte
            // aligned) stages them together with 16-byte loads: per step the
            // warp reads two elements of its 32 instances, lane l the pair of
            // instances 2 (l % 16), 2 (l % 16) + 1 of element 2 i + l / 16, and
            // stores the pair into the two owners' shared-memory columns with
            // one 16-byte store.  Otherwise every lane loads its own instance's
            // elements (8-byte loads, still coalesced across the warp).
            const int64_t k0 = __shfl_sync(FULL, cand, 0);
            const bool vec = __all_sync(FULL, want && cand == k0 + lane) && (k0 % 2 == 0) &&
                             (a.ld % 2 == 0) && ((reinterpret_cast<uintptr_t>(a.params) & 15) == 0) &&
                             k0 + THREAD_TPB <= a.batch;
            if (vec) {
                const int half = lane >> 4, pair = 2 * (lane & 15);
#pragma unroll 4
                for (int e0 = 0; e0 < E; e0 += 2) {
                    const int e = e0 + half;
                    if (e < E) {
                        const double2 v =
                            __ldg(reinterpret_cast<const double2 *>(a.params + (int64_t)e * a.ld + k0 + pair));
                        *reinterpret_cast<double2 *>(sd + e * THREAD_TPB + pair) = v;
                        if constexpr (MIXED)
                            *reinterpret_cast<float2 *>(sf + e * THREAD_TPB + pair) =
                                make_float2(float(v.x), float(v.y));
                    }
                }
                __syncwarp();
            }
            if (want && cand < a.batch) {
                k = cand;
                if (!vec) {
#pragma unroll 4
                    for (int e = 0; e < E; ++e) {
                        const double v = __ldg(a.params + (int64_t)e * a.ld + k);
                        sd[e * THREAD_TPB + lane] = v;
                        if constexpr (MIXED) sf[e * THREAD_TPB + lane] = float(v);
                    }
                }
                s.init(pv, a, k);
                got = true;
                if (s.status != ST_RUNNING) {
                    s.finish(a, k);
                    local_solved += (s.status == ST_SUCCESS);
                } else {
                    have = true;
                }
            }
            // the counter is exhausted (or the static slot is taken) once any
            // lane asked for work and got none
            exhausted = (a.counter == nullptr) || __any_sync(FULL, want && !got);
        }
        if (!__any_sync(FULL, have)) {
            if (exhausted) break;
            continue;
        }
        if (have) {
            if (a.budget_ns && global_ns() > t_end) s.status = ST_ABORTED;
            else s.pass(pv, a);
            if (s.status != ST_RUNNING) {
                s.finish(a, k);
                local_solved += (s.status == ST_SUCCESS);
                have = false;
            }
        }
    }
    if (a.solved) {
        // warp-aggregated count of solved instances
        unsigned long long t = local_solved;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
        if (lane == 0 && t) atomicAdd(a.solved, t);
    }
}

template <int N, int FAM, bool MIXED, bool ANALYTIC>
__global__ void __launch_bounds__(THREAD_TPB) k_solve_thread(SolveArgs a)
{
    thread_lanes<ThreadSolver<N, FAM, MIXED, ANALYTIC>, MIXED>(a);
}

} // namespace nls
