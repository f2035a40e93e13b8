// nls_panel.cuh -- one instance per CTA for Newton, backtracking and the
// dogleg trust region in mixed precision (FP32 Jacobian and LU), n <= 32 S,
// the Jacobian held in registers by columns.
//
// Layout.  The CTA has NW = 2 S warps.  Warp w owns the C = 16 consecutive
// columns w C .. w C + C - 1 of J; lane l of it holds rows l + 32 s (s < S)
// of those columns in registers, S x 16 floats.  Vectors (u, F, the Newton
// step, the gradient) live in shared memory, component t with thread t.
//
// LU with partial pivoting (Sec. 3.2, Fig. 5), right-looking and blocked by
// the column ownership: panel p is warp p's columns.
//  * Warp p factors its panel alone.  For each column the pivot is the
//    first position holding the largest |a_ik| over the remaining rows: each
//    lane forms (|a| + 1, ~position) keys for its rows, three warp reductions
//    give the largest key and the row holding it.  The pivot row's entries
//    reach every lane by select + shuffle from its owner, every lane scales
//    its rows' entries of the column into multipliers (published to shared
//    memory for the other warps) and updates the panel's remaining columns
//    and the right-hand side (forward substitution).  The rows' positions
//    stay in registers; no block barrier is taken inside a panel.
//  * After one CTA barrier every warp q > p applies the whole panel to its
//    columns as one rank-16 update A22 -= L21 U12: the panel's pivot rows
//    are gathered into a per-warp buffer, U12 = L11^-1 of them is formed by
//    16 lanes, and the update runs from registers with the multipliers and
//    U12 read from shared memory.  The pivot rows come out as their U12 rows,
//    the remaining rows take the update, rows eliminated before (multipliers
//    0) are untouched.  Warp p + 1 factors panel p + 1 as soon as it has
//    applied panel p, while the others still apply it.
//  * Rows never move (virtual pivoting: every row carries the position it
//    would have after the interchanges, so the pivot sequence equals an
//    explicit-swap LU's).  Back substitution walks the columns from the last
//    warp to the first: x_k = y(pivot row of k) / u_kk, then y_r -= u_rk x_k
//    for the rows r at earlier positions.
// One barrier per 16 columns, and pivot searches inside one warp, is what
// makes this faster than a 2-D block-cyclic tiling with one barrier per
// column; in FP64, where each step's FMAs must be spread over the SM's few
// FP64 units, the block-cyclic tiling (nls_cta.cuh) is kept.
//
// The factors stay in the warps' registers after the solve, so a second
// right-hand side (lu_apply: the forward elimination replayed panel by panel,
// then the back substitution) refines the Newton step when the request asks
// for it: r = -F - J dN with J in FP64, evaluated row by row from the family,
// and dN += the FP32 solve of r (classical iterative refinement).
//
// The Jacobian comes from forward-mode duals over the stencil of each row
// (Sec. 2.4), the globalisations are those of the other tilings (Sec. 2.2).
#pragma once

#include <climits>

#include "nls_common.cuh"

namespace nls {

template <int S, int C, bool MIXED>
struct PanelSmem {
    using P = typename std::conditional<MIXED, float, double>::type;
    static constexpr int NM = 32 * S;
    static constexpr int NW = NM / C;
    double u[NM], F[NM], dN[NM], ut[NM];
    P g[NM], Jg[NM], y[NM], x[NM], rdiag[NM];
    P L[2][NM][C + 1];  // a panel's multipliers by row, buffer p & 1 (padded: conflict-free)
    P part[NW][NM];     // per-warp partial row sums of J g
    alignas(16) P W[NW][C][C + 4]; // per warp: the panel's pivot rows in its columns, then U12 (rows 16-byte aligned)
    int piv[NM];        // row at position k (after the LU: the pivot row of step k)
    int rpos[NM];       // position of row r
    double rd[3][NW];
    uint64_t rm[NW];
    long long inst;
    int late;
    int singular;
};

// Pivot keys: the FP32 magnitude bits + 1 in the high half (0 = no
// candidate), the complement of the position in the low half, so the
// largest key is the largest |a_ik| at the lowest position.
NLS_DI uint64_t pivot_key(uint32_t m, int pos) { return ((uint64_t)(m + 1u) << 32) | (uint32_t)~(uint32_t)pos; }
NLS_DI int key_pos(uint64_t key) { return (int)~(uint32_t)key; }
// Warp argmax of the keys: the largest key, its position and the row (from
// the lane holding it).
NLS_DI void warp_pivot_row(uint64_t key, int row, uint32_t &kmax, int &pmin, int &prow)
{
    const uint32_t hi = __reduce_max_sync(0xffffffffu, (uint32_t)(key >> 32));
    const uint32_t lo = __reduce_max_sync(0xffffffffu, (uint32_t)(key >> 32) == hi ? (uint32_t)key : 0u);
    kmax = hi;
    pmin = (int)~lo;
    prow = (int)__reduce_max_sync(0xffffffffu, ((key >> 32) == hi && (uint32_t)key == lo && hi) ? (unsigned)row : 0u);
}
// The multipliers' reciprocal pivot: the hardware approximation (relative
// error below 2^-23, inside the FP32 LU's own rounding; a zero or non-finite
// pivot is caught before it is used).
NLS_DI float pivot_rcp(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <int S, int C, int FAM, bool MIXED>
struct PanelSolver {
    static_assert(MIXED, "the column-panel solver runs the FP32 LU of mixed precision");
    using P = typename std::conditional<MIXED, float, double>::type;
    using K = decltype(mag_bits(P(0)));
    using SM = PanelSmem<S, C, MIXED>;
    static constexpr int NM = SM::NM;
    static constexpr int NW = SM::NW;
    static constexpr int TPB = 32 * NW;

    int tid, lane, warp, n;
    int64_t B, k;
    const double *params;
    double lam; // Bratu lambda
    double fF, Delta;
    int it, nfev, rej, status, ngrad;
    bool need_jac;
    uint64_t fmag;

    NLS_DI int row(int s) const { return lane + 32 * s; }
    NLS_DI int col(int c) const { return warp * C + c; }

    // ------------------------------------------------------------ reductions
    // K block sums with one pair of barriers (warps summed in a fixed order,
    // so every thread gets the same, reproducible value)
    template <int KS>
    NLS_DI void bsumk(double (&v)[KS], SM &sm) const
    {
#pragma unroll
        for (int j = 0; j < KS; ++j) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
            if (lane == 0) sm.rd[j][warp] = v[j];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < KS; ++j) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < NW; ++w) s += sm.rd[j][w];
            v[j] = s;
        }
        __syncthreads();
    }
    // block sum of v and block max of m with one pair of barriers
    NLS_DI void bsum_max(double &v, uint64_t &m, SM &sm) const
    {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v += __shfl_xor_sync(0xffffffffu, v, o);
            const uint64_t w = __shfl_xor_sync(0xffffffffu, m, o);
            m = w > m ? w : m;
        }
        if (lane == 0) {
            sm.rd[0][warp] = v;
            sm.rm[warp] = m;
        }
        __syncthreads();
        double s = 0.0;
        uint64_t x = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            s += sm.rd[0][w];
            x = sm.rm[w] > x ? sm.rm[w] : x;
        }
        __syncthreads();
        v = s;
        m = x;
    }
    NLS_DI uint64_t bmax(uint64_t v, SM &sm) const
    {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const uint64_t w = __shfl_xor_sync(0xffffffffu, v, o);
            v = w > v ? w : v;
        }
        if (lane == 0) sm.rm[warp] = v;
        __syncthreads();
        uint64_t m = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) m = sm.rm[w] > m ? sm.rm[w] : m;
        __syncthreads();
        return m;
    }

    // ------------------------------------------------------------ residual
    // F_t(x) in FP64 for t < n, x in shared memory; returns F_t (0 for t >= n)
    NLS_DI double residual_t(const double *x) const
    {
        const int t = tid;
        if (t >= n) return 0.0;
        const double xt = x[t];
        if constexpr (FAM == FAM_CUBIC) {
            double s = 0.0;
            for (int j = 0; j < n; ++j) s = fma(__ldg(params + (int64_t)(t * n + j) * B + k), x[j], s);
            return s + xt * xt * xt - __ldg(params + (int64_t)(n * n + t) * B + k);
        } else if constexpr (FAM == FAM_BRATU) {
            const double inv_h2 = double((n + 1) * (n + 1));
            const double left = t > 0 ? x[t - 1] : 0.0;
            const double right = t < n - 1 ? x[t + 1] : 0.0;
            return inv_h2 * ((left + (-2.0) * xt) + right) + lam * exp(xt);
        } else if constexpr (FAM == FAM_SQUARE) {
            return xt * xt - __ldg(params + (int64_t)t * B + k);
        } else {
            return t == 0 ? 1.0 - xt : 10.0 * (xt - x[t - 1] * x[t - 1]);
        }
    }

    // (J(u) v)_t in FP64 at the current iterate sm.u, for t < n (0 beyond):
    // the FP64 Jacobian row of each family applied to v, evaluated on the fly
    // (no FP64 copy of J is held).  Iterative refinement's residual.
    NLS_DI double jdot64_t(const double *v, const SM &sm) const
    {
        const int t = tid;
        if (t >= n) return 0.0;
        const double ut = sm.u[t];
        if constexpr (FAM == FAM_CUBIC) {
            double s = 3.0 * ut * ut * v[t];
            for (int j = 0; j < n; ++j) s = fma(__ldg(params + (int64_t)(t * n + j) * B + k), v[j], s);
            return s;
        } else if constexpr (FAM == FAM_BRATU) {
            const double inv_h2 = double((n + 1) * (n + 1));
            const double left = t > 0 ? v[t - 1] : 0.0;
            const double right = t < n - 1 ? v[t + 1] : 0.0;
            return inv_h2 * ((left + (-2.0) * v[t]) + right) + lam * exp(ut) * v[t];
        } else if constexpr (FAM == FAM_SQUARE) {
            return 2.0 * ut * v[t];
        } else {
            return t == 0 ? -v[0] : 10.0 * (v[t] - 2.0 * sm.u[t - 1] * v[t - 1]);
        }
    }

    // ------------------------------------------------------------ Jacobian
    // this warp's C columns of J for the lane's S rows
    NLS_DI void jacobian_cols(P (&a)[S][C], const SM &sm) const
    {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int i = row(s);
            const bool live = i < n;
            const P ui = live ? P(sm.u[i]) : P(0);
            // partials of F_i over its stencil: d0 (i-1), d1 (i), d2 (i+1)
            P d0 = P(0), d1 = P(0), d2 = P(0);
            if constexpr (FAM == FAM_CUBIC) {
                const auto x = seed<1, 0, P>(ui);
                d1 = (x * x * x).d[0];
            } else if constexpr (FAM == FAM_BRATU) {
                const P inv_h2 = P((n + 1) * (n + 1));
                const auto xl = seed<3, 0, P>(P(0));
                const auto xc = seed<3, 1, P>(ui);
                const auto xr = seed<3, 2, P>(P(0));
                const auto f = inv_h2 * ((xl + P(-2) * xc) + xr) + P(lam) * exp(xc);
                d0 = f.d[0];
                d1 = f.d[1];
                d2 = f.d[2];
            } else if constexpr (FAM == FAM_SQUARE) {
                const auto x = seed<1, 0, P>(ui);
                d1 = (x * x).d[0];
            } else {
                const P ul = (live && i > 0) ? P(sm.u[i - 1]) : P(0);
                const auto xl = seed<2, 0, P>(ul);
                const auto xc = seed<2, 1, P>(ui);
                const auto f = P(10) * (xc - xl * xl);
                d0 = f.d[0];
                d1 = (i == 0) ? P(-1) : f.d[1];
            }
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const int j = col(c);
                P v = P(0);
                if (live && j < n) {
                    if constexpr (FAM == FAM_CUBIC) {
                        // linear part's coefficient, plus d(u_i^3)/du_i on the diagonal
                        v = P(__ldg(params + (int64_t)(i * n + j) * B + k));
                        if (j == i) v += d1;
                    } else {
                        // stencil families: row i depends on u_{i-1}, u_i, u_{i+1} only
                        if (j == i - 1) v = d0;
                        else if (j == i) v = d1;
                        else if (j == i + 1) v = d2;
                    }
                }
                a[s][c] = v;
            }
        }
    }

    // ------------------------------------------------------------ LU
    // Entry s_r of a per-slot array on every lane: a select chain over the
    // S slots (the slot is warp-uniform), no branch.
    NLS_DI static P pick(const P (&v)[S], int slot)
    {
        P x = v[0];
#pragma unroll
        for (int s = 1; s < S; ++s) x = (slot == s) ? v[s] : x;
        return x;
    }
    // Entry (r, cc) of this warp's columns on every lane, r = 32 slot + src.
    NLS_DI static P prow_entry(const P (&a)[S][C], int cc, int slot, int src)
    {
        P colv[S];
#pragma unroll
        for (int s = 0; s < S; ++s) colv[s] = a[s][cc];
        return __shfl_sync(0xffffffffu, pick(colv, slot), src);
    }
    // Row r's component of a per-row vector held as y[s] for rows lane + 32 s.
    NLS_DI static P vec_value(const P (&y)[S], int r)
    {
        return __shfl_sync(0xffffffffu, pick(y, r >> 5), r & 31);
    }

    // Warp `warp` factors its panel (the columns it owns) and carries the
    // right-hand side sm.y along; returns false on a zero or non-finite pivot
    // (uniform over the warp).  The positions of the lane's rows are kept in
    // registers (pos) and published to sm.rpos by their owners.
    NLS_DI bool factor_panel(P (&a)[S][C], uint32_t &rem, SM &sm, int buf) const
    {
        const K inf = inf_bits(P(0));
        P yv[S];
        int pos[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            yv[s] = row(s) < n ? sm.y[row(s)] : P(0);
            pos[s] = row(s) < n ? sm.rpos[row(s)] : INT_MAX;
        }
        bool ok = true;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int kk = col(c);
            if (kk >= n) break;
            // candidates: this lane's remaining rows (larger |a_ik| first, then
            // the lower position; a NaN below position kk is never chosen), as
            // keys (|a| bits + 1, ~position) compared as one integer
            uint64_t key[S];
#pragma unroll
            for (int s = 0; s < S; ++s) {
                K m = mag_bits(a[s][c]);
                if (pos[s] > kk && m > inf) m = K(0);
                key[s] = ((rem >> s) & 1u) ? pivot_key(m, pos[s]) : 0ull;
            }
#pragma unroll
            for (int w2 = 1; w2 < S; w2 <<= 1)
#pragma unroll
                for (int s = 0; s + w2 < S; s += 2 * w2) key[s] = key[s + w2] > key[s] ? key[s + w2] : key[s];
            int brow = -1;
#pragma unroll
            for (int s = 0; s < S; ++s)
                if (key[0] && ((rem >> s) & 1u) && pos[s] == key_pos(key[0])) brow = row(s);
            int pmin, prow;
            K kmax;
            warp_pivot_row(key[0], brow, kmax, pmin, prow);
            const int src = prow & 31, pslot = prow >> 5;
            // the pivot row's entries reach every lane by select + shuffle, each
            // just before it is used (no branch, no copy of the row held)
            if (kmax <= K(1) || kmax - K(1) >= inf) ok = false;
            const P r = pivot_rcp(prow_entry(a, c, pslot, src));
            // the pivot row leaves the remaining set; positions: it takes kk,
            // the row that held kk takes the pivot's old position
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const bool isq = pos[s] == kk, isp = (s == pslot) && (lane == src);
                if (isp) rem &= ~(1u << s);
                if (isq && !isp) {
                    pos[s] = pmin;
                    sm.rpos[row(s)] = pmin;
                }
                if (isp) {
                    pos[s] = kk;
                    sm.rpos[row(s)] = kk;
                }
            }
            // multipliers of the remaining rows (kept in column c, below the
            // row's final position) and their publication
            P l[S];
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const bool elim = (rem >> s) & 1u;
                l[s] = a[s][c] * r;
                if (elim) a[s][c] = l[s];
                sm.L[buf][row(s)][c] = elim ? l[s] : P(0);
            }
            // the rank-1 update of the panel's columns right of c, and of the
            // right-hand side
#pragma unroll
            for (int cc = 0; cc < C; ++cc) {
                if (cc <= c) continue;
                const P v = prow_entry(a, cc, pslot, src);
#pragma unroll
                for (int s = 0; s < S; ++s)
                    if ((rem >> s) & 1u) a[s][cc] -= l[s] * v;
            }
            const P yp = vec_value(yv, prow);
#pragma unroll
            for (int s = 0; s < S; ++s)
                if ((rem >> s) & 1u) yv[s] -= l[s] * yp;
            if (lane == 0) {
                sm.rdiag[kk] = r;
                sm.piv[kk] = prow;
            }
        }
#pragma unroll
        for (int s = 0; s < S; ++s)
            if (row(s) < n) sm.y[row(s)] = yv[s];
        return ok;
    }

    // Warp `warp` (> p) applies panel p to its columns as one rank-kc update
    // A22 -= L21 U12, U12 = L11^-1 (the panel's pivot rows): the pivot rows
    // come out as their U12 rows, the other remaining rows take the update,
    // rows eliminated before (multipliers 0) are untouched.
    NLS_DI void apply_panel(P (&a)[S][C], uint32_t &rem, SM &sm, int p, int buf) const
    {
        const int k0 = p * C;
        const int kc = min(C, n - k0);
        P(*W)[C + 4] = sm.W[warp];
        // the panel's pivot rows (positions k0 .. k0 + kc - 1) as they are now
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int r = row(s);
            const int pos = r < n ? sm.rpos[r] - k0 : -1;
            if (pos >= 0 && pos < kc) {
                rem &= ~(1u << s);
#pragma unroll
                for (int cc = 0; cc < C; ++cc) W[pos][cc] = a[s][cc];
            }
        }
        __syncwarp();
        // U12 = L11^-1 W, lane cc solving column cc
        if (lane < C) {
            P uc[C];
#pragma unroll
            for (int c = 0; c < C; ++c) {
                if (c < kc) {
                    const int prow = sm.piv[k0 + c];
                    P v = W[c][lane];
#pragma unroll
                    for (int c2 = 0; c2 < c; ++c2) v -= sm.L[buf][prow][c2] * uc[c2];
                    uc[c] = v;
                    W[c][lane] = v;
                }
            }
        }
        __syncwarp();
        // A -= L21 U12
        for (int c = 0; c < kc; ++c) {
            P l[S], uv[C];
#pragma unroll
            for (int s = 0; s < S; ++s) l[s] = sm.L[buf][row(s)][c];
#pragma unroll
            for (int q = 0; q < C / 4; ++q) {
                const float4 t = reinterpret_cast<const float4 *>(&W[c][0])[q];
                uv[4 * q] = t.x;
                uv[4 * q + 1] = t.y;
                uv[4 * q + 2] = t.z;
                uv[4 * q + 3] = t.w;
            }
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int cc = 0; cc < C; ++cc) a[s][cc] -= l[s] * uv[cc];
        }
        __syncwarp();
    }

    // Back substitution with the factors in a: y (by row, sm.y, already
    // forward-eliminated) to x (by column, sm.x), column by column from the
    // last warp's to the first's.
    NLS_DI void back_sub(const P (&a)[S][C], SM &sm) const
    {
        const int np = (n + C - 1) / C;
        int rp[S];
#pragma unroll
        for (int s = 0; s < S; ++s) rp[s] = row(s) < n ? sm.rpos[row(s)] : INT_MAX;
        for (int w = np - 1; w >= 0; --w) {
            if (warp == w) {
                P yv[S];
#pragma unroll
                for (int s = 0; s < S; ++s) yv[s] = row(s) < n ? sm.y[row(s)] : P(0);
#pragma unroll
                for (int c = C - 1; c >= 0; --c) {
                    const int kk = col(c);
                    if (kk >= n) continue;
                    const P xk = vec_value(yv, sm.piv[kk]) * sm.rdiag[kk];
                    if (lane == 0) sm.x[kk] = xk;
#pragma unroll
                    for (int s = 0; s < S; ++s)
                        if (rp[s] < kk) yv[s] -= a[s][c] * xk;
                }
#pragma unroll
                for (int s = 0; s < S; ++s)
                    if (row(s) < n) sm.y[row(s)] = yv[s];
            }
            __syncthreads();
        }
    }

    // A second right-hand side with the factors of lu_solve (multipliers left
    // of each row's final position in its column, U from it on; sm.piv,
    // sm.rpos, sm.rdiag): y (by row, sm.y) to x (by column, sm.x).  The
    // forward elimination replays the steps in position order, panel by
    // panel (each warp holds every row of its columns), then the back
    // substitution.
    NLS_DI void lu_apply(const P (&a)[S][C], SM &sm) const
    {
        const int np = (n + C - 1) / C;
        int rp[S];
#pragma unroll
        for (int s = 0; s < S; ++s) rp[s] = row(s) < n ? sm.rpos[row(s)] : INT_MAX;
        for (int w = 0; w < np; ++w) {
            if (warp == w) {
                P yv[S];
#pragma unroll
                for (int s = 0; s < S; ++s) yv[s] = row(s) < n ? sm.y[row(s)] : P(0);
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const int kk = col(c);
                    if (kk >= n) break;
                    const P yk = vec_value(yv, sm.piv[kk]);
#pragma unroll
                    for (int s = 0; s < S; ++s)
                        if (rp[s] > kk && rp[s] != INT_MAX) yv[s] -= a[s][c] * yk;
                }
#pragma unroll
                for (int s = 0; s < S; ++s)
                    if (row(s) < n) sm.y[row(s)] = yv[s];
            }
            __syncthreads();
        }
        back_sub(a, sm);
    }

    // Solves J x = rhs (rhs by row in sm.y, x by column to sm.x); false on a
    // zero or non-finite pivot (uniform over the CTA).
    NLS_DI bool lu_solve(P (&a)[S][C], SM &sm) const
    {
        uint32_t rem = 0;
#pragma unroll
        for (int s = 0; s < S; ++s) rem |= (row(s) < n ? 1u : 0u) << s;
        if (tid < n) {
            sm.piv[tid] = tid;
            sm.rpos[tid] = tid;
        }
        if (tid == 0) sm.singular = 0;
        __syncthreads();
        const int np = (n + C - 1) / C;
        for (int p = 0; p < np; ++p) {
            const int buf = p & 1;
            if (warp == p && !factor_panel(a, rem, sm, buf) && lane == 0) sm.singular = 1;
            __syncthreads(); // the one barrier of the panel
            if (sm.singular) return false;
            if (warp > p) apply_panel(a, rem, sm, p, buf);
        }
        back_sub(a, sm);
        return true;
    }

    // ------------------------------------------------------------ driver
    NLS_DI void set_status_from(uint64_t m, const SolveArgs &A)
    {
        fmag = m;
        if (m >= INF64_BITS) status = ST_NONFINITE;
        else if (m <= mag_bits(A.abstol)) status = ST_SUCCESS;
        else if (it >= A.maxiters) status = ST_MAXITERS;
    }

    NLS_DI void init(const SolveArgs &A, SM &sm)
    {
        if (tid < n) sm.u[tid] = A.u[(int64_t)tid * B + k];
        lam = (FAM == FAM_BRATU) ? __ldg(A.params + k) : 0.0;
        __syncthreads();
        const double f = residual_t(sm.u);
        if (tid < n) sm.F[tid] = f;
        nfev = 1;
        it = 0;
        rej = 0;
        ngrad = 0;
        Delta = TR_DELTA0;
        need_jac = true;
        status = ST_RUNNING;
        fF = f * f;
        uint64_t mx = mag_bits(f);
        bsum_max(fF, mx, sm);
        set_status_from(mx, A);
        if (status == ST_RUNNING && A.maxiters <= 0) status = ST_MAXITERS;
    }

    NLS_DI void pass(const SolveArgs &A, SM &sm)
    {
        ++it;
        if (need_jac) {
            P a[S][C];
            jacobian_cols(a, sm);
            if (tid < n) sm.y[tid] = -P(sm.F[tid]);
            __syncthreads();
            if (A.alg == ALG_TRUST_DOGLEG) {
                ++ngrad;
                // g = J^T F: each warp's columns, summed over the rows by the warp
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    P s = P(0);
#pragma unroll
                    for (int ss = 0; ss < S; ++ss)
                        if (row(ss) < n) s = fma(a[ss][c], sm.y[row(ss)], s);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                    if (lane == 0 && col(c) < n) sm.g[col(c)] = -s; // y = -F
                }
                __syncthreads();
                // J g: each warp's partial row sums over its columns, then over the warps
#pragma unroll
                for (int ss = 0; ss < S; ++ss) {
                    P s = P(0);
#pragma unroll
                    for (int c = 0; c < C; ++c)
                        if (col(c) < n) s = fma(a[ss][c], sm.g[col(c)], s);
                    sm.part[warp][row(ss)] = s;
                }
                __syncthreads();
                if (tid < n) {
                    P s = P(0);
#pragma unroll
                    for (int w = 0; w < NW; ++w) s += sm.part[w][tid];
                    sm.Jg[tid] = s;
                }
            }
            const bool ok = lu_solve(a, sm);
            if (!ok) {
                status = ST_SINGULAR;
                return;
            }
            if (tid < n) sm.dN[tid] = double(sm.x[tid]);
            __syncthreads();
            // classical iterative refinement of the Newton step: the FP64
            // residual of J dN = -F, re-solved with the same FP32 factors
            for (int r = 0; r < A.refine; ++r) {
                const double res = tid < n ? -sm.F[tid] - jdot64_t(sm.dN, sm) : 0.0;
                __syncthreads();
                if (tid < n) sm.y[tid] = P(res);
                __syncthreads();
                lu_apply(a, sm);
                if (tid < n) sm.dN[tid] += double(sm.x[tid]);
                __syncthreads();
            }
            need_jac = false;
        }
        const int t = tid;
        const bool own = t < n;
        if (A.alg == ALG_NEWTON) {
            if (own) sm.u[t] += sm.dN[t];
            __syncthreads();
            const double f = residual_t(sm.u);
            __syncthreads();
            if (own) sm.F[t] = f;
            ++nfev;
            need_jac = true;
            set_status_from(bmax(mag_bits(f), sm), A);
        } else if (A.alg == ALG_NEWTON_BACKTRACK) {
            // slope F^T J dN of Eq. 9 by linearity: J dN = -F, so it is -||F||^2
            const double s = -fF;
            const double phi0 = 0.5 * fF;
            double alpha = 1.0;
            bool ok = false;
            double f = 0.0, fFt = 0.0;
            for (int m = 0; m < LS_MAX_TRIALS; ++m) {
                if (own) sm.ut[t] = fma(alpha, sm.dN[t], sm.u[t]);
                __syncthreads();
                f = residual_t(sm.ut);
                ++nfev;
                fFt = f * f;
                uint64_t mx = mag_bits(f);
                bsum_max(fFt, mx, sm);
                if (mx < INF64_BITS && 0.5 * fFt <= phi0 + LS_C1 * alpha * s) {
                    ok = true;
                    if (own) {
                        sm.u[t] = sm.ut[t];
                        sm.F[t] = f;
                    }
                    fF = fFt;
                    __syncthreads();
                    set_status_from(mx, A);
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
            const double dn = own ? sm.dN[t] : 0.0;
            const P gt = own ? sm.g[t] : P(0), jgt = own ? sm.Jg[t] : P(0);
            const P D2 = P(Delta * Delta);
            double r3[3] = {double(P(dn) * P(dn)), double(gt * gt), double(jgt * jgt)};
            bsumk<3>(r3, sm);
            const P nN2 = P(r3[0]), gg = P(r3[1]), JgJg = P(r3[2]);
            const P tt = gg / JgJg;
            const P cc = tt * tt * gg;
            const P w = P(dn) + tt * gt;
            // the interpolation's quadratic, only when the CTA takes branch D
            // (a block-uniform decision, so the barriers inside are safe)
            P aa = P(0), bb = P(0);
            if (!(nN2 <= D2) && !(cc >= D2)) {
                double r2[2] = {double(w * w), double(-tt * gt * w)};
                bsumk<2>(r2, sm);
                aa = P(r2[0]);
                bb = P(r2[1]);
            }
            // pred = -2 F.Jd - ||Jd||^2 (Eq. 15) from block-uniform scalars:
            // J dN = -F and F.(J g) = g.g (g = J^T F), so no J d is formed
            double d, pred;
            if (nN2 <= D2) {
                d = dn;
                pred = fF;
            } else if (cc >= D2) {
                const P sc = P(Delta) / nls_sqrt(gg);
                d = double(-sc * gt);
                pred = double(sc * (P(2) * gg - sc * JgJg));
            } else {
                const P q = cc - D2;
                const P tau = (-bb + nls_sqrt(bb * bb - aa * q)) / aa;
                d = double(fma(tau, w, -tt * gt));
                const P s1 = (P(1) - tau) * tt; // J d = -s1 J g - tau F
                pred = double(s1 * (P(2) * (P(1) - tau) * gg - s1 * JgJg) + tau * (P(2) - tau) * P(fF));
            }
            if (!own) d = 0.0;
            if (own) sm.ut[t] = sm.u[t] + d;
            __syncthreads();
            const double f = residual_t(sm.ut);
            ++nfev;
            double fFt = f * f;
            uint64_t mx = mag_bits(f);
            bsum_max(fFt, mx, sm);
            const double ared = fF - fFt;
            if (tr_step_outcome(A.tr_scheme, pred > 0.0 && mx < INF64_BITS, ared, pred, !(nN2 <= D2), Delta)) {
                if (own) {
                    sm.u[t] = sm.ut[t];
                    sm.F[t] = f;
                }
                fF = fFt;
                need_jac = true;
                rej = 0;
                __syncthreads();
                set_status_from(mx, A);
            } else {
                if (++rej >= TR_MAX_REJECTIONS) {
                    status = ST_TR_STALLED;
                    return;
                }
                if (it >= A.maxiters) status = ST_MAXITERS;
            }
        }
    }

    NLS_DI void finish(const SolveArgs &A, SM &sm) const
    {
        __syncthreads();
        if (tid < n) A.u[(int64_t)tid * B + k] = sm.u[tid];
        if (tid == 0) {
            if (A.status) A.status[k] = status;
            if (A.iters) A.iters[k] = it;
            if (A.resid) A.resid[k] = bits_to_double(fmag);
            if (A.nfev) A.nfev[k] = nfev;
            if (A.ngrad) A.ngrad[k] = ngrad;
            if (A.solved && status == ST_SUCCESS) atomicAdd(A.solved, 1ull);
        }
    }
};

// columns per warp (the tile is S x 16 floats)
template <bool MIXED>
constexpr int panel_cols() { return 16; }

// CTAs per SM the register budget is sized for
template <int S, bool MIXED>
constexpr int panel_min_ctas() { return S >= 3 ? 2 : 4; }

template <int S, int C, bool MIXED>
constexpr int panel_smem_bytes()
{
    return (int)sizeof(PanelSmem<S, C, MIXED>);
}

// One instance per CTA at a time, drawn from the work counter or the static
// slot; a per-launch deadline is decided by one thread for the whole CTA.
template <int S, int C, int FAM, bool MIXED>
__global__ void __launch_bounds__(PanelSolver<S, C, FAM, MIXED>::TPB, (panel_min_ctas<S, MIXED>())) k_solve_panel(SolveArgs a)
{
    using Solver = PanelSolver<S, C, FAM, MIXED>;
    using SM = typename Solver::SM;
    apply_dyn_batch(a);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SM &sm = *reinterpret_cast<SM *>(smem_raw);
    Solver s;
    s.tid = threadIdx.x;
    s.lane = s.tid & 31;
    s.warp = s.tid >> 5;
    s.n = a.n;
    s.B = a.ld;
    s.params = a.params;
    const unsigned long long t_end = a.budget_ns ? global_ns() + a.budget_ns : ~0ull;
    bool first = true;
    for (;;) {
        if (s.tid == 0) {
            long long next;
            if (a.counter) next = (long long)atomicAdd(a.counter, 1ull);
            else next = first ? (long long)blockIdx.x : (long long)a.batch;
            sm.inst = next;
        }
        first = false;
        __syncthreads();
        s.k = sm.inst;
        __syncthreads();
        if (s.k >= a.batch) break;
        s.init(a, sm);
        while (s.status == ST_RUNNING) {
            if (a.budget_ns) {
                if (s.tid == 0) sm.late = global_ns() > t_end;
                __syncthreads();
                const bool late = sm.late;
                __syncthreads();
                if (late) {
                    s.status = ST_ABORTED;
                    break;
                }
            }
            s.pass(a, sm);
        }
        s.finish(a, sm);
    }
}

} // namespace nls
