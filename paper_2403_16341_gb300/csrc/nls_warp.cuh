// nls_warp.cuh -- one instance per warp segment of L = 8, 16 or 32 lanes,
// for n <= L (runtime n).
//
// Lane r of a segment owns component r of u and F (FP64) and row r of the
// Jacobian (FP64, or FP32 with NLS_MIXED) in registers.  Row r of J comes
// from forward-mode duals over the variables F_r depends on (Sec. 2.4: the
// stencil of F_r), scattered into the row; the cubic's linear part gives its
// coefficients directly.  The Newton system is solved with an LU with
// partial pivoting (Sec. 3.2) in which rows never move between lanes: each
// lane keeps the position its row would have after the row interchanges, so
// the pivot at step k is the first position >= k holding the largest
// |a_ik| -- the same choice as with explicit swaps.  The pivot row is
// broadcast through shared memory, the right-hand side is eliminated on the
// fly, and back substitution broadcasts one solution component per step.
//
// All segments of a warp execute each pass in lock step (idle segments run
// masked); a persistent launch refills idle segments from a work counter.
// The globalisations are those of the thread tiling: Newton (Eq. 2),
// backtracking on Eq. 8-9, dogleg trust region with Eq. 13-15.
#pragma once

#include "nls_common.cuh"

namespace nls {

constexpr int WARP_TPB = 128; // 4 warps per CTA

template <int L, bool MIXED>
struct WarpSmem {
    using P = typename std::conditional<MIXED, float, double>::type;
    double u[L];      // u broadcast (residual)
    P prow[L + 1];    // pivot row + its right-hand side
    P vec[L];         // g broadcast
    P tr[L][L + 1];   // J^T F transpose-sum
};

// Butterfly reductions inside a segment of L lanes (xor offsets < L never
// leave the segment).  `mask` names the lanes executing the call; it is a
// union of whole segments.  Every lane ends with the same bits.
template <int L, class T>
NLS_DI T seg_sum(T v, unsigned mask)
{
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}
template <int L>
NLS_DI uint64_t seg_max(uint64_t v, unsigned mask)
{
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) {
        const uint64_t w = __shfl_xor_sync(mask, v, o);
        v = w > v ? w : v;
    }
    return v;
}
template <int L>
NLS_DI uint32_t seg_max(uint32_t v, unsigned mask)
{
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(mask, v, o));
    return v;
}

template <int L, int FAM, bool MIXED>
struct WarpSolver {
    using P = typename std::conditional<MIXED, float, double>::type;
    using K = decltype(mag_bits(P(0)));
    using SM = WarpSmem<L, MIXED>;

    // ---- per-lane data of the current instance
    int r;         // row owned by this lane (0..L-1)
    int n;         // system size
    int lane0;     // first lane of the segment in the warp
    double arow[FAM == FAM_CUBIC ? L : 1];           // cubic: row r of A (FP64, residual)
    float arowf[FAM == FAM_CUBIC && MIXED ? L : 1];  // cubic, mixed: FP32 copy (Jacobian)
    double b_r;                 // cubic: b_r; square: p_r; Bratu: lambda
    double u, F, dN;
    uint64_t fmag;              // max_r |F_r| as a bit pattern (segment-uniform)
    P g, Jg, Fp;
    double fF, Delta;
    int it, nfev, rej, status;
    int ngrad; // trust region: passes that formed g = J^T F and J g
    bool need_jac;

    NLS_DI bool row_live() const { return r < n; }

    // F_r(u) in FP64; all lanes of the segment call it together
    NLS_DI double residual(const double ur, SM &sm, unsigned mask) const
    {
        double f = 0.0;
        if constexpr (FAM == FAM_CUBIC) {
            sm.u[r] = ur;
            __syncwarp(mask);
            double s = 0.0;
#pragma unroll
            for (int j = 0; j < L; ++j)
                if (j < n) s = fma(arow[j], sm.u[j], s);
            __syncwarp(mask);
            f = s + ur * ur * ur - b_r;
        } else if constexpr (FAM == FAM_BRATU) {
            const double inv_h2 = double((n + 1) * (n + 1));
            double left = __shfl_up_sync(mask, ur, 1, L);
            double right = __shfl_down_sync(mask, ur, 1, L);
            if (r == 0) left = 0.0;
            if (r >= n - 1) right = 0.0;
            f = inv_h2 * ((left + (-2.0) * ur) + right) + b_r * exp(ur);
        } else if constexpr (FAM == FAM_SQUARE) {
            f = ur * ur - b_r;
        } else {
            const double left = __shfl_up_sync(mask, ur, 1, L);
            f = (r == 0) ? 1.0 - ur : 10.0 * (ur - left * left);
        }
        return row_live() ? f : 0.0;
    }

    // row r of J(u) in precision P, by duals over the stencil of F_r
    NLS_DI void jacobian_row(P (&a)[L]) const
    {
        const P ur = P(u);
        if constexpr (FAM == FAM_CUBIC) {
            // F_r = sum_j A_rj u_j + u_r^3 - b_r: linear coefficients, then d(u_r^3)/du_r
            const auto x = seed<1, 0, P>(ur);
            const auto c = x * x * x;
#pragma unroll
            for (int j = 0; j < L; ++j) {
                P v;
                if constexpr (MIXED) v = arowf[j];
                else v = P(arow[j]);
                a[j] = (j < n) ? ((j == r) ? v + c.d[0] : v) : P(0);
            }
        } else if constexpr (FAM == FAM_BRATU) {
            const P inv_h2 = P((n + 1) * (n + 1));
            const P lam = P(b_r);
            // F_r = (u_{r-1} - 2 u_r + u_{r+1}) / h^2 + lambda e^{u_r}; seeds: 0 left, 1 centre, 2 right
            const auto xl = seed<3, 0, P>(P(0));
            const auto xc = seed<3, 1, P>(ur);
            const auto xr = seed<3, 2, P>(P(0));
            const auto f = inv_h2 * ((xl + P(-2) * xc) + xr) + lam * exp(xc);
#pragma unroll
            for (int j = 0; j < L; ++j) {
                P v = P(0);
                if (j == r - 1 && r > 0) v = f.d[0];
                if (j == r) v = f.d[1];
                if (j == r + 1 && r + 1 < n) v = f.d[2];
                a[j] = (j < n) ? v : P(0);
            }
        } else if constexpr (FAM == FAM_SQUARE) {
            const auto x = seed<1, 0, P>(ur);
            const auto f = x * x;
#pragma unroll
            for (int j = 0; j < L; ++j) a[j] = (j == r && j < n) ? f.d[0] : P(0);
        } else {
            // F_0 = 1 - u_0; F_r = 10 (u_r - u_{r-1}^2); seeds: 0 left, 1 centre
            const P ul = __shfl_up_sync(0xffffffffu, ur, 1, L); // all lanes run jacobian_row
            const auto xl = seed<2, 0, P>(ul);
            const auto xc = seed<2, 1, P>(ur);
            const auto f = P(10) * (xc - xl * xl);
#pragma unroll
            for (int j = 0; j < L; ++j) {
                P v = P(0);
                if (r == 0) v = (j == 0) ? P(-1) : P(0);
                else if (j == r - 1) v = f.d[0];
                else if (j == r) v = f.d[1];
                a[j] = (j < n) ? v : P(0);
            }
        }
        if (!row_live()) {
#pragma unroll
            for (int j = 0; j < L; ++j) a[j] = P(0);
        }
    }

    // LU with partial pivoting and on-the-fly elimination of b; on return
    // b holds x_r (component r of the solution) in lane r.  Returns false
    // (segment-uniform) on a zero or non-finite pivot.
    NLS_DI bool lu_solve(P (&a)[L], P &b, SM &sm) const
    {
        const K inf = inf_bits(P(0));
        int pos = r;              // position of this lane's row after the interchanges
        bool live = row_live();
        P rc = P(0);              // 1/pivot, kept by the lane whose row is pivot row `pos`
        bool ok = true;
#pragma unroll
        for (int k = 0; k < L; ++k) {
            if (k < n) {
                // key: |a_ik| bit pattern; NaN below the diagonal position never wins
                K m = mag_bits(a[k]);
                if (pos > k && m > inf) m = K(0);
                const bool cand = live && pos >= k;
                // larger key first, then the lower position
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
                    if (best == 0) ppos = k; // all-zero column: singular below
                }
                const bool is_piv = cand && pos == ppos;
                if (best == 0 || best >= (uint64_t)inf) ok = false;
                // broadcast the pivot row (columns > k) and its right-hand side
                if (is_piv) {
#pragma unroll
                    for (int c = k + 1; c < L; ++c) sm.prow[c] = a[c];
                    sm.prow[k] = a[k];
                    sm.prow[L] = b;
                }
                __syncwarp();
                const P piv = sm.prow[k];
                const P pr = rcp(piv);
                const P pb = sm.prow[L];
                // the row at position k moves to the pivot's old position
                if (cand && pos == k && !is_piv) pos = ppos;
                if (is_piv) {
                    pos = k;
                    rc = pr;
                }
                if (cand && !is_piv) {
                    const P l = a[k] * pr;
#pragma unroll
                    for (int c = k + 1; c < L; ++c) a[c] -= l * sm.prow[c];
                    b -= l * pb;
                }
                __syncwarp();
            }
        }
        // back substitution: x_k from the lane holding pivot row k, then
        // every lane holding an earlier pivot row removes its contribution
        P x = P(0);
#pragma unroll
        for (int k = L - 1; k >= 0; --k) {
            if (k < n) {
                P xk = P(0);
                if (live && pos == k) {
                    xk = b * rc;
                    sm.prow[0] = xk;
                }
                __syncwarp();
                xk = sm.prow[0];
                __syncwarp();
                if (r == k) x = xk;
                if (live && pos < k) b -= a[k] * xk;
            }
        }
        b = x;
        return ok;
    }

    // Load instance k and test u0; executed by the lanes in `mask` (whole segments).
    NLS_DI void init(const SolveArgs &a, int64_t k, SM &sm, unsigned mask)
    {
        const int64_t B = a.ld;
        b_r = 0.0;
        if constexpr (FAM == FAM_CUBIC) {
#pragma unroll
            for (int j = 0; j < L; ++j) {
                double v = 0.0;
                if (j < n && row_live()) v = __ldg(a.params + (int64_t)(r * n + j) * B + k);
                arow[j] = v;
                if constexpr (MIXED) arowf[j] = float(v);
            }
            if (row_live()) b_r = __ldg(a.params + (int64_t)(n * n + r) * B + k);
        } else if constexpr (FAM == FAM_BRATU) {
            b_r = __ldg(a.params + k);
        } else if constexpr (FAM == FAM_SQUARE) {
            if (row_live()) b_r = __ldg(a.params + (int64_t)r * B + k);
        }
        u = row_live() ? a.u[(int64_t)r * B + k] : 0.0;
        F = residual(u, sm, mask);
        dN = 0.0;
        nfev = 1;
        it = 0;
        rej = 0;
        ngrad = 0;
        Delta = TR_DELTA0;
        need_jac = true;
        fF = seg_sum<L>(F * F, mask);
        fmag = seg_max<L>(mag_bits(F), mask);
        if (fmag >= INF64_BITS) status = ST_NONFINITE;
        else if (fmag <= mag_bits(a.abstol)) status = ST_SUCCESS;
        else if (a.maxiters <= 0) status = ST_MAXITERS;
        else status = ST_RUNNING;
    }

    // Write instance k's results (no cross-lane communication).
    NLS_DI void finish(const SolveArgs &a, int64_t k) const
    {
        if (row_live()) a.u[(int64_t)r * a.ld + k] = u;
        if (r == 0) {
            if (a.status) a.status[k] = status;
            if (a.iters) a.iters[k] = it;
            if (a.resid) a.resid[k] = bits_to_double(fmag);
            if (a.nfev) a.nfev[k] = nfev;
            if (a.ngrad) a.ngrad[k] = ngrad;
        }
    }

    // One pass; `run` is false for idle segments, which execute the same
    // instructions (lock step) without changing their state.
    NLS_DI void pass(const SolveArgs &A, SM &sm, bool run)
    {
        if (run) ++it;
        bool failed = false;
        if (__any_sync(0xffffffffu, run && need_jac)) {
            const bool fresh = run && need_jac;
            P a[L];
            jacobian_row(a);
            const P fp = P(F);
            if (fresh) Fp = fp;
            if (A.alg == ALG_TRUST_DOGLEG) {
                // g = J^T F: column sums of F_r * row r, and J g
#pragma unroll
                for (int j = 0; j < L; ++j) sm.tr[r][j] = a[j] * fp;
                __syncwarp();
                P s = P(0);
#pragma unroll
                for (int i = 0; i < L; ++i) s += sm.tr[i][r];
                __syncwarp();
                if (fresh) g = s;
                sm.vec[r] = s;
                __syncwarp();
                P t = P(0);
#pragma unroll
                for (int j = 0; j < L; ++j) t = fma(a[j], sm.vec[j], t);
                __syncwarp();
                if (fresh) {
                    Jg = t;
                    ++ngrad;
                }
            }
            P b = -fp;
            const bool ok = lu_solve(a, b, sm);
            if (fresh) {
                if (!ok) {
                    status = ST_SINGULAR;
                    failed = true;
                } else {
                    dN = row_live() ? double(b) : 0.0;
                    need_jac = false;
                }
            }
        }
        const bool go = run && !failed;

        if (A.alg == ALG_NEWTON) {
            const double un = u + dN;
            const double Fn = residual(un, sm, 0xffffffffu);
            if (go) {
                u = un;
                F = Fn;
                ++nfev;
                need_jac = true;
            }
        } else if (A.alg == ALG_NEWTON_BACKTRACK) {
            // slope F^T J dN of Eq. 9 by linearity: J dN = -F, so it is -||F||^2
            const double s = -fF;
            const double phi0 = 0.5 * fF;
            double alpha = 1.0;
            bool trying = go, ok = false;
            for (int m = 0; m < LS_MAX_TRIALS; ++m) {
                if (!__any_sync(0xffffffffu, trying)) break;
                const double ut = fma(alpha, dN, u);
                const double Ft = residual(ut, sm, 0xffffffffu);
                const double fFt = seg_sum<L>(Ft * Ft, 0xffffffffu);
                const bool fin = seg_max<L>(mag_bits(Ft), 0xffffffffu) < INF64_BITS;
                if (trying) {
                    ++nfev;
                    if (fin && 0.5 * fFt <= phi0 + LS_C1 * alpha * s) {
                        u = ut;
                        F = Ft;
                        fF = fFt;
                        ok = true;
                        trying = false;
                    }
                }
                alpha *= LS_RHO;
            }
            if (go) {
                if (!ok) {
                    status = ST_LS_FAILED;
                    failed = true;
                } else {
                    need_jac = true;
                }
            }
        } else {
            // Every reduction is taken by all segments of the warp before any
            // per-segment branch (segments of one warp may take different
            // dogleg branches; a collective inside a branch would diverge).
            const P D2 = P(Delta * Delta);
            const P nN2 = seg_sum<L>(P(dN) * P(dN), 0xffffffffu);
            const P gg = seg_sum<L>(g * g, 0xffffffffu);
            const P JgJg = seg_sum<L>(Jg * Jg, 0xffffffffu);
            const P t = gg / JgJg; // Cauchy point c = -t g minimises the model along -g
            const P cc = t * t * gg;
            const P w = P(dN) + t * g; // dN - c
            const P aa = seg_sum<L>(w * w, 0xffffffffu);
            const P bb = seg_sum<L>(-t * g * w, 0xffffffffu);
            // pred = -2 F.Jd - ||Jd||^2 (Eq. 15) from segment-uniform scalars:
            // J dN = -F and F.(J g) = g.g (g = J^T F), so no J d is formed
            double d, pred;
            if (nN2 <= D2) {
                d = dN;
                pred = fF;
            } else if (cc >= D2) {
                const P sc = P(Delta) / nls_sqrt(gg);
                d = double(-sc * g);
                pred = double(sc * (P(2) * gg - sc * JgJg));
            } else {
                const P q = cc - D2;
                const P tau = (-bb + nls_sqrt(bb * bb - aa * q)) / aa;
                d = double(fma(tau, w, -t * g));
                const P s1 = (P(1) - tau) * t; // J d = -s1 J g - tau F
                pred = double(s1 * (P(2) * (P(1) - tau) * gg - s1 * JgJg) + tau * (P(2) - tau) * P(fF));
            }
            if (!row_live()) d = 0.0;
            const double ut = u + d;
            const double Ft = residual(ut, sm, 0xffffffffu);
            const double fFt = seg_sum<L>(Ft * Ft, 0xffffffffu);
            const bool fin = seg_max<L>(mag_bits(Ft), 0xffffffffu) < INF64_BITS;
            const double ared = fF - fFt;
            if (go) {
                ++nfev;
                if (tr_step_outcome(A.tr_scheme, pred > 0.0 && fin, ared, pred, !(nN2 <= D2), Delta)) {
                    u = ut;
                    F = Ft;
                    fF = fFt;
                    need_jac = true;
                    rej = 0;
                } else {
                    if (++rej >= TR_MAX_REJECTIONS) {
                        status = ST_TR_STALLED;
                        failed = true;
                    }
                }
            }
        }
        const uint64_t m = seg_max<L>(mag_bits(F), 0xffffffffu);
        if (run) fmag = m;
        if (go && !failed) {
            if (m >= INF64_BITS) status = ST_NONFINITE;
            else if (m <= mag_bits(A.abstol)) status = ST_SUCCESS;
            else if (it >= A.maxiters) status = ST_MAXITERS;
        }
    }
};

template <int L, bool MIXED>
constexpr int warp_smem_bytes()
{
    return (WARP_TPB / 32) * (32 / L) * (int)sizeof(WarpSmem<L, MIXED>);
}

// The segment loop shared by the warp-tiled solvers S (r, n, lane0, status,
// init / pass / finish): segments take instances from the work counter (or
// the static slot), every pass runs in lock step over the whole warp.
template <class S, int L, bool MIXED>
NLS_DI void warp_lanes(SolveArgs &a)
{
    apply_dyn_batch(a);
    using SM = WarpSmem<L, MIXED>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int SEGS = 32 / L;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int seg = lane / L;
    SM &sm = reinterpret_cast<SM *>(smem_raw)[warp * SEGS + seg];
    const unsigned FULL = 0xffffffffu;

    const unsigned long long t_end = a.budget_ns ? global_ns() + a.budget_ns : ~0ull;
    S s;
    s.r = lane % L;
    s.n = a.n;
    s.lane0 = seg * L;
    s.status = ST_ABORTED;
    bool have = false, exhausted = false, first = true;
    int64_t k = -1;
    unsigned long long local_solved = 0;
    const int64_t warp_global = (int64_t)blockIdx.x * (WARP_TPB / 32) + warp;

    for (;;) {
        // segments are the units of work: one ballot bit per segment leader
        const unsigned seg_live = __ballot_sync(FULL, have && s.r == 0);
        const int live = __popc(seg_live);
        if (!exhausted && live <= (SEGS > 1 ? SEGS - 1 : 0)) {
            const bool want = !have;
            int64_t cand = a.batch;
            if (a.counter == nullptr) {
                if (first && want) cand = warp_global * SEGS + seg;
            } else {
                const unsigned m = __ballot_sync(FULL, want && s.r == 0);
                const int leader = m ? __ffs(m) - 1 : 0;
                unsigned long long base = 0;
                if (lane == leader && m) base = atomicAdd(a.counter, (unsigned long long)__popc(m));
                base = __shfl_sync(FULL, base, leader);
                if (want) cand = (int64_t)base + __popc(m & ((1u << (seg * L)) - 1u));
            }
            first = false;
            const bool got = want && cand < a.batch;
            // the lanes of segments that got an instance load it together
            const unsigned gm = __ballot_sync(FULL, got);
            if (got) {
                k = cand;
                s.init(a, k, sm, gm);
                if (s.status != ST_RUNNING) {
                    s.finish(a, k);
                    local_solved += (s.status == ST_SUCCESS && s.r == 0);
                } else {
                    have = true;
                }
            }
            exhausted = (a.counter == nullptr) || __any_sync(FULL, want && !got);
        }
        if (!__any_sync(FULL, have)) {
            if (exhausted) break;
            continue;
        }
        // the deadline test is warp-uniform (lane 0's clock), so skipping the
        // pass never splits a collective
        const bool late = a.budget_ns && __shfl_sync(FULL, global_ns(), 0) > t_end;
        if (late) {
            if (have) s.status = ST_ABORTED;
        } else {
            s.pass(a, sm, have);
        }
        if (have && s.status != ST_RUNNING) {
            s.finish(a, k);
            local_solved += (s.status == ST_SUCCESS && s.r == 0);
            have = false;
        }
    }
    if (a.solved) {
        unsigned long long t = local_solved;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
        if (lane == 0 && t) atomicAdd(a.solved, t);
    }
}

template <int L, int FAM, bool MIXED>
__global__ void __launch_bounds__(WARP_TPB) k_solve_warp(SolveArgs a)
{
    warp_lanes<WarpSolver<L, FAM, MIXED>, L, MIXED>(a);
}

} // namespace nls
