// nls_cta.cuh -- one instance per CTA, for 32 < n <= 128 (any n <= 16 R).
//
// 256 threads form a 16 x 16 grid.  Thread (ty, tx) keeps, in registers,
// the R x R block-cyclic tile of the Jacobian with rows ty + 16 a and
// columns tx + 16 b (a, b < R), in FP64 or (NLS_MIXED) FP32, so the rank-1
// updates of the LU run out of registers at FMA rate; only the pivot
// column's multipliers and the pivot row cross threads, through shared
// memory.  Vectors (u, F, the Newton step, the gradient) live in shared
// memory, component t with thread t.
//
// LU with partial pivoting (Sec. 3.2), rows never move: every row carries
// the position it would have after the interchanges, and the pivot at step
// k is the first position >= k holding the largest |a_ik| (the choice an
// explicit-swap LU makes).  Step k: the 16 owners of column k (one
// half-warp) reduce their candidates (redux.sync on 32-bit halves of the
// keys), write the multipliers and publish the pivot; after the step's one
// barrier every thread takes the pivot row's entries of its columns by
// shuffles and updates its tile.  After each block of 16 steps the block's
// pivot rows are compacted into one tile slot, which the later steps skip.
// The right-hand side is eliminated alongside; back substitution walks the
// positions down.
// This tiling serves the FP64 Newton-family solves (mixed precision takes the
// column-panel kernel of nls_panel.cuh), and the NEXT-4 solvers and the
// adjoint in both precisions.
//
// The Jacobian tile comes from forward-mode duals over the stencil of each
// owned row (Sec. 2.4).  The globalisations are those of the other tilings.
#pragma once

#include <climits>

#include "nls_common.cuh"

namespace nls {

constexpr int CTA_T = 16;
constexpr int CTA_TPB = CTA_T * CTA_T;
constexpr int CTA_NMAX = 128;

template <bool MIXED>
struct CtaSmem {
    using P = typename std::conditional<MIXED, float, double>::type;
    double u[CTA_NMAX], F[CTA_NMAX], dN[CTA_NMAX], ut[CTA_NMAX], Ft[CTA_NMAX];
    P Fp[CTA_NMAX], g[CTA_NMAX], Jg[CTA_NMAX], rhs[CTA_NMAX];
    P lcol[2][CTA_NMAX];    // multipliers of step k in buffer k & 1
    P rdiag[CTA_NMAX], x[CTA_NMAX];
    P red[CTA_T][CTA_NMAX]; // partial sums of J^T F and J g
    int pos_row[CTA_NMAX];  // row holding pivot position k
    int row_pos[CTA_NMAX];  // position of row i after the interchanges so far
    int qidx[CTA_NMAX];     // compaction after block b: 16 b + pair index of a moving row
    uint64_t ckey[2];       // pivot of step k in slot k & 1: key, position, row
    int cpos[2], crow[2];
    double rd[3][CTA_TPB / 32];
    uint64_t rm[CTA_TPB / 32];
    long long inst;
    int late;
};

// Adds the factor U in pivot-position order, for the single-warp back
// substitution (row stride NM + 1: a column walk hits 32 different banks).
template <bool MIXED, int NM>
struct CtaSmemU : CtaSmem<MIXED> {
    typename CtaSmem<MIXED>::P U[NM][NM + 1];
};

template <int R, int FAM, bool MIXED>
struct CtaSolver {
    using P = typename std::conditional<MIXED, float, double>::type;
    using K = decltype(mag_bits(P(0)));
    static constexpr int NM = CTA_T * R;
    using SM = CtaSmemU<MIXED, NM>;
    // the LU's compaction stages 32 rows in the space of U (unused until the
    // factorisation ends)
    static_assert(NM * (NM + 1) >= 2 * CTA_T * NM, "compaction buffer");

    int tid, ty, tx, lane, warp, n;
    int64_t B, k;
    const double *params;
    double lam; // Bratu lambda
    double fF, Delta;
    int it, nfev, rej, status;
    int ngrad; // trust region: passes that formed g = J^T F and J g
    bool need_jac;
    uint64_t fmag;

    NLS_DI int row(int a) const { return ty + CTA_T * a; }
    NLS_DI int col(int b) const { return tx + CTA_T * b; }
    // bit a: row(a) < n
    NLS_DI uint32_t exist_mask() const
    {
        uint32_t m = 0;
#pragma unroll
        for (int a = 0; a < R; ++a) m |= (row(a) < n ? 1u : 0u) << a;
        return m;
    }

    // ------------------------------------------------------------ reductions
    // K block sums with one pair of barriers (warps summed in a fixed order,
    // so every thread gets the same, reproducible value)
    template <int K>
    NLS_DI void bsumk(double (&v)[K], SM &sm) const
    {
#pragma unroll
        for (int j = 0; j < K; ++j) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
            if (lane == 0) sm.rd[j][warp] = v[j];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < K; ++j) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < CTA_TPB / 32; ++w) s += sm.rd[j][w];
            v[j] = s;
        }
        __syncthreads();
    }
    NLS_DI double bsum(double v, SM &sm) const
    {
        double a[1] = {v};
        bsumk<1>(a, sm);
        return a[0];
    }
    NLS_DI float bsum(float v, SM &sm) const { return float(bsum(double(v), sm)); }
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
        for (int w = 0; w < CTA_TPB / 32; ++w) {
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
        for (int w = 0; w < CTA_TPB / 32; ++w) m = sm.rm[w] > m ? sm.rm[w] : m;
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

    // ------------------------------------------------------------ Jacobian tile
    NLS_DI void jacobian_tile(P (&a)[R][R], const SM &sm) const
    {
#pragma unroll
        for (int aa = 0; aa < R; ++aa) {
            const int i = row(aa);
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
            for (int bb = 0; bb < R; ++bb) {
                const int j = col(bb);
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
                a[aa][bb] = v;
            }
        }
    }

    // ------------------------------------------------------------ LU
    // Solves J x = rhs (rhs in sm.rhs, x to sm.x); returns false on a zero or
    // non-finite pivot (uniform over the CTA).  The 16 owners of column k are
    // one half-warp (tx = tid / 16), so the pivot candidates are reduced with
    // shuffles; every thread then reads the single winner.
    template <bool COMPACT = true>
    NLS_DI bool lu_solve(P (&a)[R][R], SM &sm) const
    {
        const K inf = inf_bits(P(0));
        // bit aa: row(aa) exists and is not a pivot row yet
        uint32_t remmask = exist_mask();
        if (tid < n) {
            sm.row_pos[tid] = tid; // position of row tid
            sm.pos_row[tid] = tid; // row at position tid
            if (COMPACT) sm.qidx[tid] = -1;
        }
        __syncthreads();
        bool ok = true;
#pragma unroll
        for (int b = 0; b < R; ++b) {
            // slots below lo hold pivot rows only (after the compaction below)
            const int lo = COMPACT ? b : 0;
            for (int c = 0; c < CTA_T; ++c) {
                const int kk = CTA_T * b + c;
                if (kk >= n) break;
                const int par = kk & 1;
                if (tx == c) {
                    // the owners of column kk: local best over their remaining rows
                    // (larger |a_ik| first, then the lower position) ...
                    uint64_t best = 0;
                    int bpos = INT_MAX, brow = -1;
                    P bval = P(0);
#pragma unroll
                    for (int aa = lo; aa < R; ++aa) {
                        if (!((remmask >> aa) & 1u)) continue;
                        const int i = row(aa);
                        const int pi = sm.row_pos[i];
                        K m = mag_bits(a[aa][b]);
                        if (pi > kk && m > inf) m = K(0);
                        if (brow < 0 || (uint64_t)m > best || ((uint64_t)m == best && pi < bpos)) {
                            best = m;
                            bpos = pi;
                            brow = i;
                            bval = a[aa][b];
                        }
                    }
                    // ... reduced over the half-warp with redux.sync on 32-bit
                    // halves (largest high word, then the largest low word
                    // among its holders, then the lowest position among the
                    // holders of the largest key): one exact 64-bit argmax
                    const unsigned hm = 0xFFFFu << (16 * (c & 1));
                    uint64_t kmax;
                    int pmin;
                    if constexpr (sizeof(K) == 4) {
                        // 32-bit magnitudes: (|a| + 1, complement of the position) in
                        // one key, so its maximum gives the pivot and its position
                        const uint32_t kh = brow >= 0 ? (uint32_t)best + 1u : 0u;
                        const uint32_t kl = brow >= 0 ? ~(uint32_t)bpos : 0u;
                        const uint32_t H = __reduce_max_sync(hm, kh);
                        const uint32_t L = __reduce_max_sync(hm, kh == H ? kl : 0u);
                        kmax = H;
                        pmin = H ? (int)~L : INT_MAX;
                    } else {
                        const uint64_t key = brow >= 0 ? best + 1 : 0; // +1: a valid zero key beats no candidate
                        const uint32_t kh = (uint32_t)(key >> 32), kl = (uint32_t)key;
                        const uint32_t H = __reduce_max_sync(hm, kh);
                        const uint32_t L = __reduce_max_sync(hm, kh == H ? kl : 0u);
                        kmax = ((uint64_t)H << 32) | L;
                        pmin = __reduce_min_sync(hm, (brow >= 0 && key == kmax) ? bpos : INT_MAX);
                    }
                    const unsigned wb = __ballot_sync(hm, brow >= 0 && bpos == pmin);
                    const int src = wb ? __ffs(wb) - 1 : (16 * (c & 1));
                    const P pv = __shfl_sync(hm, bval, src);
                    const int prow_i = __shfl_sync(hm, brow, src);
                    const P r = rcp(pv);
                    // ... which then write the multipliers of their rows and the pivot
#pragma unroll
                    for (int aa = lo; aa < R; ++aa) {
                        const int i = row(aa);
                        const bool elim = ((remmask >> aa) & 1u) && i != prow_i;
                        const P l = a[aa][b] * r;
                        if (i < n) sm.lcol[par][i] = elim ? l : P(0);
                        // the multiplier stays in column kk of its row (below the
                        // row's final position, so lu_apply finds it in sm.U)
                        if (elim) a[aa][b] = l;
                    }
                    if (lane == src) {
                        sm.ckey[par] = kmax ? kmax - 1 : 0;
                        sm.cpos[par] = pmin;
                        sm.crow[par] = prow_i;
                        sm.rdiag[kk] = r;
                        // interchange: the pivot row takes position kk, the row that
                        // held kk takes the pivot's old position
                        const int q = sm.pos_row[kk];
                        sm.row_pos[q] = pmin;
                        sm.pos_row[pmin] = q;
                        sm.row_pos[prow_i] = kk;
                        sm.pos_row[kk] = prow_i;
                    }
                }
                __syncthreads(); // the one barrier of the step
                const uint64_t best = sm.ckey[par];
                const int prow_i = sm.crow[par];
                if (best == 0 || best >= (uint64_t)inf) ok = false;
                const int tp = prow_i & (CTA_T - 1); // ty of the pivot row's owners
                const int ap = prow_i / CTA_T;       // ... and its slot in their tiles
                const uint32_t rem = remmask & ~(ty == tp ? 1u << ap : 0u);
                // the pivot row's entries of this thread's columns sit in lane tp of
                // its half-warp (same tx): width-16 shuffles, slot chosen by a
                // CTA-uniform switch
                P pr[R];
#pragma unroll
                for (int bb = 0; bb < R; ++bb) pr[bb] = P(0);
                switch (ap) {
#define NLS_PROW_CASE(A)                                                                          \
    case A:                                                                                       \
        if (A < R && A >= lo) {                                                                   \
            _Pragma("unroll") for (int bb = b; bb < R; ++bb) if (!COMPACT || CTA_T * bb < n) pr[bb] = \
                __shfl_sync(0xffffffffu, a[A < R ? A : 0][bb], tp, CTA_T);                        \
        }                                                                                         \
        break;
                    NLS_PROW_CASE(0) NLS_PROW_CASE(1) NLS_PROW_CASE(2) NLS_PROW_CASE(3)
                    NLS_PROW_CASE(4) NLS_PROW_CASE(5) NLS_PROW_CASE(6) NLS_PROW_CASE(7)
#undef NLS_PROW_CASE
                }
                remmask = rem;
#pragma unroll
                for (int aa = lo; aa < R; ++aa) {
                    if (!((rem >> aa) & 1u)) continue;
                    const P l = sm.lcol[par][row(aa)];
#pragma unroll
                    for (int bb = b; bb < R; ++bb) {
                        if (COMPACT && CTA_T * bb >= n) break; // CTA-uniform: no columns left
                        if (bb > b || tx > c) a[aa][bb] -= l * pr[bb];
                    }
                }
                if (tid < n && tid >= CTA_T * lo && tid != prow_i)
                    sm.rhs[tid] -= sm.lcol[par][tid] * sm.rhs[prow_i];
                // the next barrier orders these reads before buffer `par` is reused
            }
            // Compaction, which leaves every result unchanged (a row carries its
            // position, multipliers and right-hand side): after the 16 steps of
            // block b, the block's pivot rows that sit outside slot b trade
            // places with the rows of slot b that are not pivots, so that slot b
            // holds exactly the block's pivot rows and the later steps skip it
            // as a whole.  The row update work drops from all R slots per step to
            // the R - b live ones.
            if (COMPACT && b + 1 < R && CTA_T * (b + 1) < n) {
                __syncthreads(); // the block's last update and bookkeeping are done
                if (warp == 0) {
                    // lanes 0..15: the pivot row of position 16 b + j; lanes 16..31:
                    // row 16 b + j of slot b.  The q-th mover of each half pairs up
                    // with the q-th mover of the other.
                    const int j = lane & (CTA_T - 1);
                    const bool outer = lane < CTA_T;
                    const int r = outer ? sm.pos_row[CTA_T * b + j] : CTA_T * b + j;
                    const bool mv = outer ? (r / CTA_T != b) : (sm.row_pos[r] >= CTA_T * (b + 1));
                    const unsigned bal = __ballot_sync(0xffffffffu, mv);
                    const unsigned mine = outer ? (bal & 0xFFFFu) : (bal >> CTA_T);
                    const int q = __popc(mine & ((1u << j) - 1u));
                    if (mv) {
                        sm.qidx[r] = CTA_T * b + q;
                        if (outer) {
                            unsigned o = bal >> CTA_T;
                            for (int t = 0; t < q; ++t) o &= o - 1u;
                            const int ra = CTA_T * b + __ffs(o) - 1; // its partner in slot b
                            const int pb = CTA_T * b + j;             // position of row r
                            const int pa = sm.row_pos[ra];
                            const P hb = sm.rhs[r], ha = sm.rhs[ra];
                            sm.row_pos[ra] = pb;
                            sm.pos_row[pb] = ra;
                            sm.rhs[ra] = hb;
                            sm.row_pos[r] = pa;
                            sm.pos_row[pa] = r;
                            sm.rhs[r] = ha;
                        }
                    }
                }
                __syncthreads();
                // rows of slot b to stage rows 0..15, the pivot rows to 16..31
                P *stage = &sm.U[0][0];
#pragma unroll
                for (int aa = b; aa < R; ++aa) {
                    const int qv = row(aa) < n ? sm.qidx[row(aa)] : -1;
                    if ((qv >> 4) == b) {
                        P *st = stage + ((aa == b ? 0 : CTA_T) + (qv & (CTA_T - 1))) * NM;
#pragma unroll
                        for (int bb = 0; bb < R; ++bb) st[col(bb)] = a[aa][bb];
                    }
                }
                __syncthreads();
#pragma unroll
                for (int aa = b; aa < R; ++aa) {
                    const int qv = row(aa) < n ? sm.qidx[row(aa)] : -1;
                    if ((qv >> 4) == b) {
                        const P *st = stage + ((aa == b ? CTA_T : 0) + (qv & (CTA_T - 1))) * NM;
#pragma unroll
                        for (int bb = 0; bb < R; ++bb) a[aa][bb] = st[col(bb)];
                    }
                }
                remmask = exist_mask() & ~((2u << b) - 1u);
            }
        }
        __syncthreads();
        // L \ U in pivot-position order: U on and right of each row's position
        // (the back substitution), its multipliers left of it (lu_apply)
#pragma unroll
        for (int aa = 0; aa < R; ++aa) {
            if (row(aa) >= n) continue;
            const int pa = sm.row_pos[row(aa)];
#pragma unroll
            for (int bb = 0; bb < R; ++bb)
                if (col(bb) < n) sm.U[pa][col(bb)] = a[aa][bb];
        }
        __syncthreads();
        // back substitution by warp 0: lane l keeps the right-hand sides of
        // positions l, l + 32, ...; one shuffle broadcasts x_k per step
        if (warp == 0) {
            constexpr int J = (NM + 31) / 32;
            P y[J];
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const int p = lane + 32 * j;
                y[j] = p < n ? sm.rhs[sm.pos_row[p]] : P(0);
            }
            for (int kk = n - 1; kk >= 0; --kk) {
                const int jk = kk >> 5;
                P yk = P(0);
#pragma unroll
                for (int j = 0; j < J; ++j) yk = (j == jk) ? y[j] : yk;
                const P xk = __shfl_sync(0xffffffffu, yk * sm.rdiag[kk], kk & 31);
                if (lane == 0) sm.x[kk] = xk;
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const int p = lane + 32 * j;
                    if (p < kk) y[j] -= sm.U[p][kk] * xk;
                }
            }
        }
        __syncthreads();
        return ok;
    }

    // One warp's solve with the factors lu_solve left in sm.U (multipliers
    // left of each row's position, U from it on), sm.pos_row and sm.rdiag:
    // y holds the right-hand side by position (lane l: positions l, l + 32,
    // ...); forward substitution over the positions (the replay of the
    // right-hand-side elimination), then the back substitution, one shuffle
    // broadcast per step; x (by column) goes to xout.  Warp-synchronous.
    static constexpr int YJ = (NM + 31) / 32;
    NLS_DI void lu_apply_warp(const SM &sm, P (&y)[YJ], P *xout) const
    {
        for (int c = 0; c < n; ++c) {
            const int jc = c >> 5;
            P yc = P(0);
#pragma unroll
            for (int j = 0; j < YJ; ++j) yc = (j == jc) ? y[j] : yc;
            yc = __shfl_sync(0xffffffffu, yc, c & 31);
#pragma unroll
            for (int j = 0; j < YJ; ++j) {
                const int p = lane + 32 * j;
                if (p > c && p < n) y[j] -= sm.U[p][c] * yc;
            }
        }
        for (int kk = n - 1; kk >= 0; --kk) {
            const int jk = kk >> 5;
            P yk = P(0);
#pragma unroll
            for (int j = 0; j < YJ; ++j) yk = (j == jk) ? y[j] : yk;
            const P xk = __shfl_sync(0xffffffffu, yk * sm.rdiag[kk], kk & 31);
            if (lane == 0) xout[kk] = xk;
#pragma unroll
            for (int j = 0; j < YJ; ++j) {
                const int p = lane + 32 * j;
                if (p < kk) y[j] -= sm.U[p][kk] * xk;
            }
        }
    }

    // x = A^-1 rhs (sm.rhs by row, sm.x by column) on warp 0.
    NLS_DI void lu_apply(SM &sm) const
    {
        __syncthreads();
        if (warp == 0) {
            P y[YJ];
#pragma unroll
            for (int j = 0; j < YJ; ++j) {
                const int p = lane + 32 * j;
                y[j] = p < n ? sm.rhs[sm.pos_row[p]] : P(0);
            }
            lu_apply_warp(sm, y, sm.x);
        }
        __syncthreads();
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
            P a[R][R];
            jacobian_tile(a, sm);
            if (tid < n) sm.Fp[tid] = P(sm.F[tid]);
            __syncthreads();
            if (A.alg == ALG_TRUST_DOGLEG) {
                ++ngrad;
                // g = J^T F and J g
#pragma unroll
                for (int bb = 0; bb < R; ++bb) {
                    P s = P(0);
#pragma unroll
                    for (int aa = 0; aa < R; ++aa)
                        if (row(aa) < n) s = fma(a[aa][bb], sm.Fp[row(aa)], s);
                    if (col(bb) < CTA_NMAX) sm.red[ty][col(bb)] = s;
                }
                __syncthreads();
                if (tid < n) {
                    P s = P(0);
#pragma unroll
                    for (int q = 0; q < CTA_T; ++q) s += sm.red[q][tid];
                    sm.g[tid] = s;
                }
                __syncthreads();
#pragma unroll
                for (int aa = 0; aa < R; ++aa) {
                    P s = P(0);
#pragma unroll
                    for (int bb = 0; bb < R; ++bb)
                        if (col(bb) < n) s = fma(a[aa][bb], sm.g[col(bb)], s);
                    sm.red[tx][row(aa)] = s;
                }
                __syncthreads();
                if (tid < n) {
                    P s = P(0);
#pragma unroll
                    for (int q = 0; q < CTA_T; ++q) s += sm.red[q][tid];
                    sm.Jg[tid] = s;
                }
            }
            if (tid < n) sm.rhs[tid] = -sm.Fp[tid];
            __syncthreads();
            const bool ok = lu_solve(a, sm);
            if (!ok) {
                status = ST_SINGULAR;
                return;
            }
            if (tid < n) sm.dN[tid] = double(sm.x[tid]);
            __syncthreads();
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

template <bool MIXED, int R>
constexpr int cta_smem_bytes()
{
    return (int)sizeof(CtaSmemU<MIXED, CTA_T * R>);
}

// The instance loop shared by the CTA-tiled solvers S (tid ... params set
// here; init / pass / finish; a status): one instance per CTA at a time,
// drawn from the work counter or the static slot.
template <class S>
NLS_DI void cta_loop(SolveArgs &a)
{
    apply_dyn_batch(a);
    using SM = typename S::SM;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SM &sm = *reinterpret_cast<SM *>(smem_raw);
    S s;
    s.tid = threadIdx.x;
    s.tx = s.tid / CTA_T; // the 16 owners of a column form one half-warp
    s.ty = s.tid % CTA_T;
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
                // one clock for the whole CTA: the decision stays uniform
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

template <int R, int FAM, bool MIXED>
__global__ void __launch_bounds__(CTA_TPB) k_solve_cta(SolveArgs a)
{
    cta_loop<CtaSolver<R, FAM, MIXED>>(a);
}

} // namespace nls
