// nls_common.cuh -- shared device definitions: launch arguments, status
// codes, bit-exact FP64 tests on integer pipes, the residual families.
#pragma once

#include <cstdint>
#include <type_traits>

#include "nls_dual.cuh"

namespace nls {

enum : int { FAM_CUBIC = 0, FAM_BRATU = 1, FAM_SQUARE = 2, FAM_ROSENBROCK = 3 };
enum : int {
    ALG_NEWTON = 0,
    ALG_NEWTON_BACKTRACK = 1,
    ALG_TRUST_DOGLEG = 2,
    ALG_POTRA_PTAK = 4,
    ALG_HALLEY = 5,
    ALG_BROYDEN = 6,
    ALG_MOD_BROYDEN = 7
};
enum : int {
    ST_RUNNING = -1,
    ST_SUCCESS = 0,
    ST_MAXITERS = 1,
    ST_SINGULAR = 2,
    ST_NONFINITE = 3,
    ST_LS_FAILED = 4,
    ST_TR_STALLED = 5,
    ST_ABORTED = 6
};

// Backtracking (Sec. 2.2.1) and trust-region (Sec. 2.2.2) constants; the
// paper gives no values, these are the readings documented in nls.h.
constexpr double LS_C1 = 1e-4;
constexpr double LS_RHO = 0.5;
constexpr int LS_MAX_TRIALS = 30;
constexpr double TR_DELTA0 = 1.0;
constexpr double TR_ETA_EXPAND = 0.75;
constexpr double TR_GROW = 2.0;
constexpr double TR_SHRINK = 0.25;
constexpr double TR_DELTA_MAX = 1e3;
constexpr int TR_MAX_REJECTIONS = 32;
// NocedalWright radius update (Nocedal & Wright, Numerical Optimization,
// Algorithm 4.1; Tab. 3): acceptance threshold eta
constexpr double TR_NW_ETA = 1e-4;
enum : int { TR_SIMPLE = 0, TR_NOCEDAL_WRIGHT = 1 };

// Everything one launch needs for one uniform-size group of instances.
struct SolveArgs {
    const double *params; // [E][ld]
    double *u;            // [n][ld], u0 in, iterate out
    int64_t batch;        // instances solved: k = 0 .. batch-1
    int64_t ld;           // leading dimension (row stride) of params and u, >= batch
    int n;
    int alg;
    double abstol;
    int maxiters;
    int32_t *status;
    int32_t *iters;
    double *resid;
    int32_t *nfev;
    int32_t *ngrad;              // trust region: passes that formed g = J^T F (may be null)
    unsigned long long *solved;  // += #SUCCESS (may be null)
    unsigned long long *counter; // work counter for persistent launches (null = static)
    int refill_below;            // persistent: refill idle lanes when live lanes <= this
    // when set, the instance count is min(batch, *dyn_batch), read on the
    // device (a count produced by an earlier kernel of the same stream)
    const unsigned long long *dyn_batch;
    // > 0: stop iterating once this many nanoseconds of %globaltimer have
    // passed since the kernel started; unfinished instances end NLS_ABORTED
    unsigned long long budget_ns;
    int tr_scheme; // TR_SIMPLE or TR_NOCEDAL_WRIGHT
    // mixed precision, CTA tiling: iterative-refinement steps per Newton
    // solve (r = -F - J64 dN in FP64, re-solved with the FP32 factors); 0: none
    int refine;
};

// Outcome of one trust-region trial step (Sec. 2.2.2, Eq. 15): returns
// whether the step is accepted and updates the radius.  ok: pred > 0 and
// F(u + d) finite (otherwise rho = -inf); boundary: the dogleg step ended on
// the region's boundary (branch C or D).  With pred > 0 every comparison of
// rho = ared / pred with a threshold is ared against threshold * pred, so no
// FP64 divide is taken.
//   Simple: accept iff rho > 0; then double (capped) iff rho > 3/4;
//           on rejection shrink to Delta / 4.
//   NocedalWright: shrink to Delta / 4 iff rho < 1/4; else double (capped)
//           iff rho > 3/4 and the step reached the boundary; accept iff
//           rho > eta, independently of the radius change.
NLS_DI bool tr_step_outcome(int scheme, bool ok, double ared, double pred, bool boundary, double &Delta)
{
    if (scheme == TR_NOCEDAL_WRIGHT) {
        if (!ok || ared < 0.25 * pred) Delta *= TR_SHRINK;
        else if (boundary && ared > TR_ETA_EXPAND * pred) Delta = fmin(TR_GROW * Delta, TR_DELTA_MAX);
        return ok && ared > TR_NW_ETA * pred;
    }
    if (ok && ared > 0.0) {
        if (ared > TR_ETA_EXPAND * pred) Delta = fmin(TR_GROW * Delta, TR_DELTA_MAX);
        return true;
    }
    Delta *= TR_SHRINK;
    return false;
}

NLS_DI unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

NLS_DI void apply_dyn_batch(SolveArgs &a)
{
    if (a.dyn_batch) {
        const long long d = (long long)*a.dyn_batch;
        if (d < a.batch) a.batch = d;
    }
}

// ---------------------------------------------------------------------------
// Bit-exact FP64 tests on the integer pipes.  On GB300 the FP64 pipe is the
// scarce resource (about 2 DFMA per clock per SM), so comparisons that only
// decide convergence or finiteness are done on the IEEE bit patterns: for
// non-NaN doubles, |x| <= |y| iff the sign-cleared bit patterns compare the
// same way as unsigned integers; NaN patterns are above +Inf's.
constexpr uint64_t INF64_BITS = 0x7FF0000000000000ull;
constexpr uint32_t INF32_BITS = 0x7F800000u;

NLS_DI uint64_t mag_bits(double x) { return (uint64_t)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull; }
NLS_DI uint32_t mag_bits(float x) { return __float_as_uint(x) & 0x7FFFFFFFu; }
NLS_DI uint64_t inf_bits(double) { return INF64_BITS; }
NLS_DI uint32_t inf_bits(float) { return INF32_BITS; }

// max_i |v_i| as a bit pattern (a NaN anywhere gives a pattern above Inf).
template <int N>
NLS_DI uint64_t max_mag_bits(const double (&v)[N])
{
    uint64_t m = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) m = max(m, mag_bits(v[i]));
    return m;
}

NLS_DI double bits_to_double(uint64_t b) { return __longlong_as_double((long long)b); }

NLS_DI double rcp(double x) { return __drcp_rn(x); }
NLS_DI float rcp(float x) { return __frcp_rn(x); }
NLS_DI double nls_sqrt(double x) { return __dsqrt_rn(x); }
NLS_DI float nls_sqrt(float x) { return __fsqrt_rn(x); }

template <int I, int N, class Fn>
NLS_DI void static_for(Fn &&f)
{
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, N>(f);
    }
}

// ---------------------------------------------------------------------------
// Parameter view: one instance's parameters, element e at sd[e * stride]
// (FP64) and its FP32 copy at sf[e * stride] (mixed precision only).
struct ParamView {
    const double *sd;
    const float *sf;
    int stride;
    template <class T>
    NLS_DI T get(int e) const
    {
        if constexpr (std::is_same<T, double>::value) return sd[e * stride];
        else return sf[e * stride];
    }
};

// Vector accessors for a compile-time size N: plain values (residual) or
// seeded duals (Jacobian by forward mode).
template <int N, class T>
struct PlainVec {
    using scalar = T;
    const T *x;
    template <int J>
    NLS_DI T get() const { return x[J]; }
};

template <int N, class T>
struct SeedVec {
    using scalar = T;
    const T *x;
    template <int J>
    NLS_DI Dual<N, (1u << J), T> get() const { return seed<N, J, T>(x[J]); }
};

// Jets along the direction a at the point x (second directional derivative).
template <int N, class T>
struct JetVec {
    using scalar = T;
    const T *x;
    const T *a;
    template <int J>
    NLS_DI Jet<T, false> get() const { return Jet<T, false>{x[J], a[J], T(0)}; }
};

// ---------------------------------------------------------------------------
// Residual families, written once over the scalar type: row<I>(p, u) is the
// I-th component F_I(u; p); with SeedVec it is a dual whose partials are
// row I of the Jacobian.  jac_analytic writes the closed-form Jacobian.
template <int FAM, int N>
struct Family;

// F_i = sum_j A_ij u_j + u_i^3 - b_i; parameters A (row-major) then b.
template <int N>
struct Family<FAM_CUBIC, N> {
    static constexpr int E = N * N + N;
    template <int I, int J, class PV, class U, class Acc>
    NLS_DI static auto dot(const PV &p, const U &u, const Acc &acc)
    {
        using T = typename U::scalar;
        if constexpr (J == N) return acc;
        else return dot<I, J + 1>(p, u, acc + p.template get<T>(I * N + J) * u.template get<J>());
    }
    // The sum starts from A_i0 u_0 - b_i, so every term of the row is one
    // fused multiply-add: N + 1 FP64 FMAs and one multiply per row.
    template <int I, class PV, class U>
    NLS_DI static auto row(const PV &p, const U &u)
    {
        using T = typename U::scalar;
        auto s = dot<I, 1>(p, u, p.template get<T>(I * N) * u.template get<0>() - p.template get<T>(N * N + I));
        return s + cube(u.template get<I>());
    }
    template <class T, class PV>
    NLS_DI static void jac_analytic(const PV &p, const T (&u)[N], T (&J)[N][N])
    {
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j = 0; j < N; ++j) J[i][j] = p.template get<T>(i * N + j);
#pragma unroll
        for (int i = 0; i < N; ++i) J[i][i] += T(3) * u[i] * u[i];
    }
};

// 1-D Bratu: F_i = (u_{i-1} - 2 u_i + u_{i+1}) / h^2 + lambda e^{u_i}, h = 1/(N+1),
// zero Dirichlet boundaries; 1/h^2 is the exact integer (N+1)^2.
template <int N>
struct Family<FAM_BRATU, N> {
    static constexpr int E = 1;
    template <int I, class PV, class U>
    NLS_DI static auto row(const PV &p, const U &u)
    {
        using T = typename U::scalar;
        const T inv_h2 = T((N + 1) * (N + 1));
        const T lam = p.template get<T>(0);
        auto ui = u.template get<I>();
        auto c = T(-2) * ui;
        auto l = [&] {
            if constexpr (I > 0) return u.template get<I - 1>() + c;
            else return c;
        }();
        auto s = [&] {
            if constexpr (I < N - 1) return l + u.template get<I + 1>();
            else return l;
        }();
        return inv_h2 * s + lam * exp(ui);
    }
    template <class T, class PV>
    NLS_DI static void jac_analytic(const PV &p, const T (&u)[N], T (&J)[N][N])
    {
        const T inv_h2 = T((N + 1) * (N + 1));
        const T lam = p.template get<T>(0);
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j = 0; j < N; ++j)
                J[i][j] = (j == i - 1 || j == i + 1) ? inv_h2 : T(0);
#pragma unroll
        for (int i = 0; i < N; ++i) J[i][i] = T(-2) * inv_h2 + lam * exp(u[i]);
    }
};

// F_i = u_i^2 - p_i (the Sec. 2.3 example)
template <int N>
struct Family<FAM_SQUARE, N> {
    static constexpr int E = N;
    template <int I, class PV, class U>
    NLS_DI static auto row(const PV &p, const U &u)
    {
        using T = typename U::scalar;
        auto ui = u.template get<I>();
        return ui * ui - p.template get<T>(I);
    }
    template <class T, class PV>
    NLS_DI static void jac_analytic(const PV &, const T (&u)[N], T (&J)[N][N])
    {
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j = 0; j < N; ++j) J[i][j] = (i == j) ? T(2) * u[i] : T(0);
    }
};

// generalized Rosenbrock, Eq. 5: F_1 = 1 - u_1, F_i = 10 (u_i - u_{i-1}^2)
template <int N>
struct Family<FAM_ROSENBROCK, N> {
    static constexpr int E = 0;
    template <int I, class PV, class U>
    NLS_DI static auto row(const PV &, const U &u)
    {
        using T = typename U::scalar;
        if constexpr (I == 0) return T(1) - u.template get<0>();
        else {
            auto a = u.template get<I - 1>();
            return T(10) * (u.template get<I>() - a * a);
        }
    }
    template <class T, class PV>
    NLS_DI static void jac_analytic(const PV &, const T (&u)[N], T (&J)[N][N])
    {
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j = 0; j < N; ++j) J[i][j] = T(0);
        J[0][0] = T(-1);
#pragma unroll
        for (int i = 1; i < N; ++i) {
            J[i][i] = T(10);
            J[i][i - 1] = T(-20) * u[i - 1];
        }
    }
};

template <int FAM>
constexpr int family_params(int n)
{
    return FAM == FAM_CUBIC ? n * n + n : FAM == FAM_BRATU ? 1 : FAM == FAM_SQUARE ? n : 0;
}

} // namespace nls
